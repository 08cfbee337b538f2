"""The conjugate-gradient placement loop (optimizer = FFTPL_OPT_CG) on the
GPU against the oracle's CG loop: the first 10 iterations on the bounds of
test_gpu_loop.py (positions 1e-4 relative L2; W~, HPWL, N, lambda 1e-4
relative; tau 1e-4 absolute; the step, chosen by a line search through two
evaluations, 1e-3), in both reduction modes, and a run to the overflow
target whose iteration count and final HPWL stay close to the oracle's.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1312_4587_gb300 import fftpl
    fftpl.lib()
    return fftpl


def run_gpu(F, inst, iters, **opts):
    import torch
    with F.Problem(inst, optimizer=F.FFTPL_OPT_CG, **opts) as p:
        x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        rows, ran = F.fftpl_step(p.h, iters)
        x = torch.empty_like(x0); y = torch.empty_like(y0)
        F.fftpl_place_positions(p.h, x, y)
        F.fftpl_check(p.h)
        return x.cpu().numpy(), y.cpu().numpy(), rows, ran


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


@pytest.mark.parametrize("det", [0, 1])
def test_cg_first_iterations_match_oracle(F, det):
    inst = synth.make_instance("tiny")
    ox, oy, orows, oran = oracle.cg(inst, 10, gamma_fixed=inst.gamma)
    gx, gy, grows, gran = run_gpu(F, inst, 10, gamma_fixed=inst.gamma, deterministic=det)
    assert gran == oran == 10
    assert rel(np.concatenate([gx, gy]), np.concatenate([ox, oy])) < 1e-4
    for k in range(10):
        for key, rtol, atol in (("hpwl", 1e-4, 0), ("W", 1e-4, 0), ("N", 1e-4, 0),
                                ("lam", 1e-4, 0), ("tau", 0, 1e-4), ("alpha", 1e-3, 0)):
            a, b = grows[k][key], orows[k][key]
            assert abs(a - b) <= rtol * abs(b) + atol, (k, key, a, b)


def test_cg_reaches_target_like_oracle(F):
    inst = synth.make_instance("tiny")
    _, _, orows, oran = oracle.cg(inst, 400, gamma_fixed=0.0, stop_on_tau=True)
    _, _, grows, gran = run_gpu(F, inst, 400, gamma_fixed=0.0, stop_on_tau=1)
    assert gran < 400 and grows[-1]["tau"] <= 0.1
    # a nonlinear iteration: FP32 and FP64 runs need not stop at the same
    # iteration, but they stop close together and at a similar wirelength
    assert abs(gran - oran) <= max(5, 0.2 * oran)
    assert grows[-1]["hpwl"] == pytest.approx(orows[-1]["hpwl"], rel=0.1)


def test_cg_state_round_trip(F):
    """Saving and restoring the loop state mid-run continues the same run."""
    import torch
    inst = synth.make_instance("tiny")
    with F.Problem(inst, optimizer=F.FFTPL_OPT_CG, gamma_fixed=inst.gamma, deterministic=1) as p:
        x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        F.fftpl_step(p.h, 5)
        blob = F.fftpl_state_save(p.h)
        a, _ = F.fftpl_step(p.h, 5)
        F.fftpl_state_load(p.h, blob)
        b, _ = F.fftpl_step(p.h, 5)
    assert [r["hpwl"] for r in a] == [r["hpwl"] for r in b]
