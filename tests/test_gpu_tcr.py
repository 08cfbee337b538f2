"""Radix tensor-core solve path (solve_path FFTPL_SOLVE_TC_RADIX): every
complex DFT of the transform path as two small dense products on tcgen05
(64-point and n/64-point DFT blocks, bf16 x 3 split, FP32 accumulation),
against the FP64 oracle with the tensor-core bound (2e-4 relative L2 on
psi, E_x, E_y, grad N and N); the outputs that do not depend on the solve
path keep the transform path's bounds.  n = 256 (16 rows per second-stage
tile), 512, 1024 and, sampled, 2048 and 4096 (one row per tile)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_TC = 2e-4


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
        out.update(gNx=g[0].cpu().numpy(), gNy=g[1].cpu().numpy(), gWx=g[2].cpu().numpy(),
                   gWy=g[3].cpu().numpy(), rep=rep)
        F.fftpl_check(p.h)
    return out


def errors(got, ref):
    return {
        "rho": rel(got["rho"], ref["rho"]),
        "psi": rel(got["psi"], ref["psi"]),
        "ex": rel(got["ex"], ref["ex"]),
        "ey": rel(got["ey"], ref["ey"]),
        "gN": rel(np.concatenate([got["gNx"], got["gNy"]]), np.concatenate([ref["gNx"], ref["gNy"]])),
        "gW": rel(np.concatenate([got["gWx"], got["gWy"]]), np.concatenate([ref["gWx"], ref["gWy"]])),
        "N": abs(got["rep"]["N"] - ref["N"]) / abs(ref["N"]),
        "hpwl": abs(got["rep"]["hpwl"] - ref["hpwl"]) / abs(ref["hpwl"]),
        "tau": abs(got["rep"]["tau"] - ref["tau"]) / max(abs(ref["tau"]), 1e-12),
    }


LIMITS = {"rho": 1e-6, "psi": TOL_TC, "ex": TOL_TC, "ey": TOL_TC, "gN": TOL_TC, "gW": 1e-5,
          "N": TOL_TC, "hpwl": 1e-6, "tau": 1e-5}


@pytest.mark.parametrize("name", ["precision_sub", "large"])
@pytest.mark.parametrize("det", [0, 1])
def test_tcr_eval_parity(F, name, det):
    inst = synth.make_instance(name)
    ref = oracle.eval_instance(inst, maps=True)
    got = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_RADIX, deterministic=det)
    errs = errors(got, ref)
    print("radix tensor-core path errors", name, {k: f"{v:.2e}" for k, v in errs.items()})
    bad = {k: (errs[k], LIMITS[k]) for k in errs if not errs[k] <= LIMITS[k]}
    assert not bad, f"parity failures {bad}"


def test_tcr_random_cells_1024(F):
    """n = 1024 (4 rows per second-stage tile): 30000 random cells."""
    rng = np.random.default_rng(1024)
    inst = synth.make_instance("tiny")
    m, L = 30000, 1536.0
    x, y, w, h = synth.random_cells(rng, m, (0.0, 0.0, L, L), wmax=4.0, hmax=2.0)
    inst.n = 1024
    inst.region = (0.0, 0.0, L, L)
    inst.m_mov, inst.m_fix = m, 0
    inst.w, inst.h, inst.x, inst.y = w, h, x, y
    inst.fix_x = np.zeros(0, np.float32); inst.fix_y = np.zeros(0, np.float32)
    inst.net_ptr = np.array([0, 2], np.int32); inst.pin_cell = np.array([0, 1], np.int32)
    inst.pin_dx = np.zeros(2, np.float32); inst.pin_dy = np.zeros(2, np.float32)
    ref = oracle.eval_instance(inst, maps=True)
    got = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_RADIX)
    errs = errors(got, ref)
    for k in ("psi", "ex", "ey", "gN", "N"):
        assert errs[k] < TOL_TC, (k, errs[k])


@pytest.mark.parametrize("name,n_samples", [("precision", 64)])
def test_tcr_full_size_sampled(F, name, n_samples):
    """2048 x 2048 bins, 2.2M cells: psi, E at sampled bins against the
    oracle's series, every map against the transform path."""
    inst = synth.make_instance(name)
    n, m = inst.n, inst.m_mov
    t = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_RADIX)
    rho, _, _ = oracle.density(inst.region, n, inst.target_density, inst.x, inst.y,
                               inst.w[:m], inst.h[:m], inst.fix_x, inst.fix_y, inst.w[m:],
                               inst.h[m:])
    a = oracle.dct_coeffs(rho)
    rng = np.random.default_rng(7)
    xs = rng.integers(0, n, n_samples); ys = rng.integers(0, n, n_samples)
    psi, ex, ey = oracle.potential_at(a, inst.region[2] - inst.region[0],
                                      inst.region[3] - inst.region[1], xs, ys)
    for k, ref in (("psi", psi), ("ex", ex), ("ey", ey)):
        assert rel(t[k][ys, xs], ref) < TOL_TC, k
    f = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_FFT)
    for k in ("psi", "ex", "ey"):
        assert rel(t[k], f[k]) < TOL_TC, k
    assert abs(t["rep"]["N"] - f["rep"]["N"]) / abs(f["rep"]["N"]) < TOL_TC
    assert t["rep"]["tau"] == pytest.approx(f["rep"]["tau"], rel=1e-6)


def test_tcr_largest_grid(F):
    """n = 4096 (one row per second-stage tile, 64-point DFTs both ways)."""
    rng = np.random.default_rng(4096)
    inst = synth.make_instance("tiny")
    m, L = 20000, 2048.0
    x, y, w, h = synth.random_cells(rng, m, (0.0, 0.0, L, L), wmax=3.0, hmax=3.0)
    inst.n = 4096
    inst.region = (0.0, 0.0, L, L)
    inst.m_mov, inst.m_fix = m, 0
    inst.w, inst.h, inst.x, inst.y = w, h, x, y
    inst.fix_x = np.zeros(0, np.float32); inst.fix_y = np.zeros(0, np.float32)
    inst.net_ptr = np.array([0, 2], np.int32); inst.pin_cell = np.array([0, 1], np.int32)
    inst.pin_dx = np.zeros(2, np.float32); inst.pin_dy = np.zeros(2, np.float32)
    t = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_RADIX)
    f = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_FFT)
    for k in ("psi", "ex", "ey"):
        assert rel(t[k], f[k]) < TOL_TC, k
    assert t["rep"]["N"] == pytest.approx(f["rep"]["N"], rel=TOL_TC)


def test_tcr_rejects_small_grid(F):
    inst = synth.make_instance("medium")   # n = 128
    with pytest.raises(F.FFTPLError) as e:
        F.Problem(inst, solve_path=F.FFTPL_SOLVE_TC_RADIX)
    assert e.value.status == F.FFTPL_EINVAL
