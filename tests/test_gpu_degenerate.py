"""Degenerate instances against the oracle: no nets, no movable cells (fixed
cells and their nets only), every cell outside the region, and the smallest
grids (n = 16 and 32), in both reduction modes, on the default bounds."""
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


def variant(**kw):
    base = synth.make_instance("tiny")
    d = dict(base.__dict__)
    d.update(kw)
    return synth.Instance(**d)


def no_movable():
    base = synth.make_instance("tiny")
    w = np.array([4, 6, 3], np.float32); h = np.array([4, 2, 3], np.float32)
    return synth.Instance(name="no_movable", region=base.region, n=base.n, target_density=1.0,
                          gamma=base.gamma, m_mov=0, m_fix=3, w=w, h=h,
                          fix_x=np.array([20, 60, 100], np.float32),
                          fix_y=np.array([30, 70, 90], np.float32),
                          net_ptr=np.array([0, 2, 3], np.int32),
                          pin_cell=np.array([0, 1, 2], np.int32),
                          pin_dx=np.zeros(3, np.float32), pin_dy=np.zeros(3, np.float32),
                          x=np.zeros(0, np.float32), y=np.zeros(0, np.float32))


CASES = {
    "no_nets": lambda: variant(net_ptr=np.zeros(1, np.int32), pin_cell=np.zeros(0, np.int32),
                               pin_dx=np.zeros(0, np.float32), pin_dy=np.zeros(0, np.float32)),
    "outside": lambda: (lambda b: variant(x=b.x + 1000.0, y=b.y + 1000.0))(synth.make_instance("tiny")),
    "n16": lambda: variant(n=16),
    "n32": lambda: variant(n=32),
    "no_movable": no_movable,
}


def rel(a, b):
    a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / nb) if nb > 0 else float(np.abs(a).max(initial=0.0))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("det", [0, 1])
def test_degenerate_eval(F, case, det):
    import torch
    inst = CASES[case]()
    ref = oracle.eval_instance(inst, maps=True)
    with F.Problem(inst, deterministic=det) as p:
        xd = torch.from_numpy(np.ascontiguousarray(inst.x)).cuda()
        yd = torch.from_numpy(np.ascontiguousarray(inst.y)).cuda()
        g = [torch.empty_like(xd) for _ in range(4)]
        rep = F.fftpl_eval(p.h, xd, yd, inst.gamma, *g)
        fl = {k: v.cpu().numpy() for k, v in F.fftpl_fields(p.h, inst.n).items()}
        F.fftpl_check(p.h)
    for k in ("rho", "psi", "ex", "ey"):
        assert rel(fl[k], ref[k]) < 1e-5, k
    if inst.m_mov:
        g = [t.cpu().numpy() for t in g]
        assert rel(np.concatenate(g[:2]), np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5
        assert rel(np.concatenate(g[2:]), np.concatenate([ref["gWx"], ref["gWy"]])) < 1e-5
    for key, tol in (("N", 2e-6), ("W", 1e-6), ("hpwl", 1e-6)):
        assert rep[key] == pytest.approx(ref[key], rel=tol, abs=1e-9), key
    assert rep["tau"] == pytest.approx(ref["tau"], abs=1e-6)


def test_no_movable_cells_cannot_be_placed(F):
    import torch
    with F.Problem(no_movable()) as p:
        e = torch.zeros(0, device="cuda")
        with pytest.raises(F.FFTPLError) as ei:
            F.fftpl_place_init(p.h, e, e)
        assert ei.value.status == F.FFTPL_EINVAL
        assert F.fftpl_bin_ranges(p.h, e, e, torch.zeros(0, dtype=torch.int32, device="cuda")) == 0
