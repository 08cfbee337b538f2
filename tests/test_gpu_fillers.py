"""Fillers on the GPU: instances extended by the filler rule's cells (pin-less
movable cells) evaluate and iterate like any other instance, against the
oracle on the default bounds (relative L2 1e-5 for maps and gradients, 1e-6
for W~ and HPWL, 2e-6 for N; the loop's first 10 iterations as in
test_gpu_loop.py)."""
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


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def extended(F, name):
    inst = synth.make_instance(name)
    cnt, fw, fh = F.fftpl_fillers(inst.region, inst.w, inst.h, inst.m_mov, inst.fix_x,
                                  inst.fix_y, inst.target_density)
    assert cnt > 0
    return synth.with_fillers(inst, cnt, fw, fh)


@pytest.mark.parametrize("name", ["medium", "precision_sub"])
@pytest.mark.parametrize("det", [0, 1])
def test_eval_with_fillers(F, name, det):
    import torch
    inst = extended(F, name)
    ref = oracle.eval_instance(inst, maps=True)
    with F.Problem(inst, deterministic=det) as p:
        xd = torch.from_numpy(inst.x).cuda(); yd = torch.from_numpy(inst.y).cuda()
        g = [torch.empty_like(xd) for _ in range(4)]
        rep = F.fftpl_eval(p.h, xd, yd, inst.gamma, *g)
        fl = {k: v.cpu().numpy() for k, v in F.fftpl_fields(p.h, inst.n).items()}
    g = [t.cpu().numpy() for t in g]
    for k in ("rho", "psi", "ex", "ey"):
        assert rel(fl[k], ref[k]) < 1e-5, k
    assert rel(np.concatenate(g[:2]), np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5
    assert rel(np.concatenate(g[2:]), np.concatenate([ref["gWx"], ref["gWy"]])) < 1e-5
    # fillers carry no pins: zero wirelength gradient
    m0 = inst.m_mov - inst.extra["fillers"]
    assert np.all(g[2][m0:] == 0) and np.all(g[3][m0:] == 0)
    assert rep["N"] == pytest.approx(ref["N"], rel=2e-6)
    assert rep["W"] == pytest.approx(ref["W"], rel=1e-6)


def test_loop_with_fillers(F):
    import torch
    inst = extended(F, "tiny")
    ox, oy, orows, oran = oracle.nesterov(inst, 10, gamma_fixed=inst.gamma)
    with F.Problem(inst, gamma_fixed=inst.gamma) as p:
        x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        grows, gran = F.fftpl_step(p.h, 10)
        gx = torch.empty_like(x0); gy = torch.empty_like(y0)
        F.fftpl_place_positions(p.h, gx, gy)
    assert gran == oran == 10
    assert rel(np.concatenate([gx.cpu().numpy(), gy.cpu().numpy()]), np.concatenate([ox, oy])) < 1e-4
    for k in range(10):
        for key, rtol, atol in (("hpwl", 1e-4, 0), ("N", 1e-4, 0), ("tau", 0, 1e-4)):
            a, b = grows[k][key], orows[k][key]
            assert abs(a - b) <= rtol * abs(b) + atol, (k, key, a, b)
