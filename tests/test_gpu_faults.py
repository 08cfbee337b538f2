"""Failure handling made on the host (no GPU fault is provoked): injected
allocation failures, calls in the wrong state, bad arguments on live
handles."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1312_4587_gb300 import fftpl
    fftpl.lib()
    return fftpl


def test_injected_allocation_failures_leak_nothing(F):
    import torch
    inst = synth.make_instance("medium")
    # warm up the context and a full create/destroy cycle
    with F.Problem(inst, deterministic=1):
        pass
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    failures = 0
    for k in range(1, 40):
        F.fftpl_debug_fail_alloc_after(k)
        try:
            with F.Problem(inst, deterministic=1):
                pass
        except F.FFTPLError as e:
            assert e.status == F.FFTPL_ENOMEM
            assert "injected" in F.fftpl_last_error(None)
            failures += 1
        finally:
            F.fftpl_debug_fail_alloc_after(0)
    assert failures >= 10
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0


def test_wrong_state_and_bad_arguments(F):
    import torch
    inst = synth.make_instance("tiny")
    with F.Problem(inst) as p:
        with pytest.raises(F.FFTPLError) as e:
            F.fftpl_step(p.h, 3)
        assert e.value.status == F.FFTPL_ESTATE
        with pytest.raises(F.FFTPLError) as e:
            F.fftpl_fields(p.h, inst.n)
        assert e.value.status == F.FFTPL_ESTATE
        x = torch.from_numpy(inst.x).cuda(); y = torch.from_numpy(inst.y).cuda()
        with pytest.raises(F.FFTPLError) as e:
            F.fftpl_wa(p.h, x, y, -1.0)
        assert e.value.status == F.FFTPL_EINVAL
        with pytest.raises(F.FFTPLError) as e:
            F.fftpl_state_load(p.h, b"\0" * 64)
        assert e.value.status == F.FFTPL_EINVAL
        # the handle still works after the errors
        assert F.fftpl_density(p.h, x, y) > 0
        F.fftpl_check(p.h)


def test_no_device_wait_can_time_out(F):
    """The kernels contain no device-side waits; the error word stays clear
    through a full evaluation and a loop run."""
    import torch
    inst = synth.make_instance("tiny")
    with F.Problem(inst) as p:
        x = torch.from_numpy(inst.x).cuda(); y = torch.from_numpy(inst.y).cuda()
        F.fftpl_eval(p.h, x, y, inst.gamma)
        F.fftpl_place_init(p.h, x, y)
        F.fftpl_step(p.h, 5)
        F.fftpl_check(p.h)
