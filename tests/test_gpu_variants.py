"""Model variants on the GPU against the oracle: the LSE wirelength
(wirelength = FFTPL_WL_LSE) and the Helmholtz smoothing of Eq. 4
(helmholtz_eps > 0), on both solve paths and in the placement loop.

Tolerances are those of the default model on the same path: relative L2
1e-5 for the maps and gradients on the transform path (2e-4 on the
tensor-core path), 1e-6 relative for the FP64 sums of float32 per-net terms
(W~, HPWL), 2e-6 for N; the loop's first 10 iterations as in
test_gpu_loop.py.
"""
import math

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
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(a - b) / (nb if nb > 0 else 1.0))


def gpu_eval(F, inst, **opts):
    import torch
    with F.Problem(inst, **opts) as p:
        xd = torch.from_numpy(inst.x).cuda(); yd = torch.from_numpy(inst.y).cuda()
        g = [torch.empty_like(xd) for _ in range(4)]
        rep = F.fftpl_eval(p.h, xd, yd, inst.gamma, *g)
        fl = F.fftpl_fields(p.h, inst.n)
        out = {k: v.cpu().numpy() for k, v in fl.items()}
        out.update(gN=np.concatenate([g[0].cpu().numpy(), g[1].cpu().numpy()]),
                   gW=np.concatenate([g[2].cpu().numpy(), g[3].cpu().numpy()]), rep=rep)
        F.fftpl_check(p.h)
    return out


def eps_for(inst, k=4.0):
    """A Helmholtz term comparable to the k-th lowest mode's w^2."""
    L = inst.region[2] - inst.region[0]
    return k * (math.pi / L) ** 2


@pytest.mark.parametrize("name", ["tiny", "medium", "precision_sub", "large"])
@pytest.mark.parametrize("det", [0, 1])
def test_lse_eval_parity(F, name, det):
    inst = synth.make_instance(name)
    ref = oracle.eval_instance(inst, wirelength=oracle.WL_LSE)
    got = gpu_eval(F, inst, wirelength=F.FFTPL_WL_LSE, deterministic=det)
    assert rel(got["gW"], np.concatenate([ref["gWx"], ref["gWy"]])) < 1e-5
    assert rel(got["gN"], np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5
    assert got["rep"]["W"] == pytest.approx(ref["W"], rel=1e-6)
    assert got["rep"]["hpwl"] == pytest.approx(ref["hpwl"], rel=1e-6)
    assert got["rep"]["gW_l1"] == pytest.approx(ref["gW_l1"], rel=1e-5)


@pytest.mark.parametrize("name", ["tiny", "medium", "precision_sub"])
@pytest.mark.parametrize("det", [0, 1])
def test_helmholtz_eval_parity(F, name, det):
    inst = synth.make_instance(name)
    eps = eps_for(inst)
    ref = oracle.eval_instance(inst, maps=True, helmholtz_eps=eps)
    got = gpu_eval(F, inst, helmholtz_eps=eps, deterministic=det)
    for k in ("psi", "ex", "ey"):
        assert rel(got[k], ref[k]) < 1e-5, k
    assert rel(got["gN"], np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5
    assert got["rep"]["N"] == pytest.approx(ref["N"], rel=2e-6)


@pytest.mark.parametrize("name", ["medium", "precision_sub"])
def test_helmholtz_tensor_core_parity(F, name):
    inst = synth.make_instance(name)
    eps = eps_for(inst)
    ref = oracle.eval_instance(inst, maps=True, helmholtz_eps=eps)
    got = gpu_eval(F, inst, helmholtz_eps=eps, solve_path=F.FFTPL_SOLVE_TC_BF16X3)
    for k in ("psi", "ex", "ey"):
        assert rel(got[k], ref[k]) < 2e-4, k
    assert rel(got["gN"], np.concatenate([ref["gNx"], ref["gNy"]])) < 2e-4
    assert got["rep"]["N"] == pytest.approx(ref["N"], rel=2e-4)


def test_eps_zero_is_poisson_and_bad_options_rejected(F):
    inst = synth.make_instance("tiny")
    # deterministic mode: bit-reproducible, so "the same as the default" is exact
    a = gpu_eval(F, inst, deterministic=1)
    b = gpu_eval(F, inst, helmholtz_eps=0.0, wirelength=F.FFTPL_WL_WA, deterministic=1)
    for k in ("psi", "ex", "ey", "gN", "gW"):
        assert np.array_equal(a[k], b[k]), k
    for bad in (dict(helmholtz_eps=-1.0), dict(helmholtz_eps=float("inf")),
                dict(wirelength=5)):
        with pytest.raises(F.FFTPLError) as ei:
            F.Problem(inst, **bad)
        assert ei.value.status == F.FFTPL_EINVAL


@pytest.mark.parametrize("variant", ["lse", "helmholtz"])
def test_loop_first_iterations(F, variant):
    import torch
    inst = synth.make_instance("tiny")
    if variant == "lse":
        okw, gkw = dict(wirelength=oracle.WL_LSE), dict(wirelength=F.FFTPL_WL_LSE)
    else:
        e = eps_for(inst)
        okw, gkw = dict(helmholtz_eps=e), dict(helmholtz_eps=e)
    ox, oy, orows, oran = oracle.nesterov(inst, 10, gamma_fixed=inst.gamma, **okw)
    with F.Problem(inst, gamma_fixed=inst.gamma, **gkw) as p:
        x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        grows, gran = F.fftpl_step(p.h, 10)
        gx = torch.empty_like(x0); gy = torch.empty_like(y0)
        F.fftpl_place_positions(p.h, gx, gy)
    assert gran == oran == 10
    assert rel(np.concatenate([gx.cpu().numpy(), gy.cpu().numpy()]), np.concatenate([ox, oy])) < 1e-4
    for k in range(10):
        for key, rtol, atol in (("hpwl", 1e-4, 0), ("W", 1e-4, 0), ("N", 1e-4, 0),
                                ("lam", 1e-4, 0), ("tau", 0, 1e-4)):
            a, b = grows[k][key], orows[k][key]
            assert abs(a - b) <= rtol * abs(b) + atol, (k, key, a, b)
