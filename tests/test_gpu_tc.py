"""Tensor-core solve path (solve_path FFTPL_SOLVE_TC_BF16X3).

The GEMM core first, through fftpl_debug_tc_gemm:
  * integer-valued bf16 operands, whose products and float32 sums are exact,
    so that any misplaced element (descriptor, swizzle, TMEM lane/column,
    stage ring) shows as a bit difference against numpy;
  * random operands split into hi + lo, within the float32 accumulation
    bound of the exact product;
  * the bounded-wait path: a launch that issues no operand loads returns
    with the error word set and its output untouched.
Then the whole evaluation against the FP64 oracle, relative L2:
  psi, E_x, E_y, grad N <= 2e-4 and N <= 2e-4 (bf16 x 3 products keep about
  16 bits of each operand: 2^-16 relative per product, four dependent
  contractions); the other outputs do not depend on the solve path and keep
  the transform path's bounds.
"""
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


def bf16(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).to(torch.bfloat16).cuda()


def run_gemm(F, ah, al, bh, bl, nsplit=3, no_loads=0, fill=0.0):
    import torch
    M, N = ah.shape[0], bh.shape[0]
    d = torch.full((M, N), fill, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    F.fftpl_debug_tc_gemm(ah, al, bh, bl, d, err, nsplit=nsplit, no_loads=no_loads)
    torch.cuda.synchronize()
    return d.cpu().numpy(), int(err.item())


@pytest.mark.parametrize("M,N,K", [(128, 128, 64), (256, 384, 192), (384, 256, 512),
                                   (128, 128, 320), (128, 256, 1024)])
def test_gemm_integer_exact(F, M, N, K):
    """Small integers: every partial sum is an integer below 2^24, exact in
    float32, so the tensor-core result equals the FP64 product bit for bit."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    ah = rng.integers(-6, 7, (M, K)).astype(np.float32)
    al = rng.integers(-2, 3, (M, K)).astype(np.float32)
    bh = rng.integers(-6, 7, (N, K)).astype(np.float32)
    bl = rng.integers(-2, 3, (N, K)).astype(np.float32)
    d3, e3 = run_gemm(F, bf16(ah), bf16(al), bf16(bh), bf16(bl), 3)
    d1, e1 = run_gemm(F, bf16(ah), bf16(al), bf16(bh), bf16(bl), 1)
    A = ah.astype(np.float64); B = bh.astype(np.float64)
    ref3 = A @ B.T + A @ bl.astype(np.float64).T + al.astype(np.float64) @ B.T
    ref1 = A @ B.T
    assert e3 == 0 and e1 == 0
    assert np.array_equal(d3.astype(np.float64), ref3)
    assert np.array_equal(d1.astype(np.float64), ref1)


def test_gemm_split_accuracy(F):
    """Random float32 operands split as x = hi + lo: the three-product sum is
    within the float32 accumulation bound plus the dropped lo*lo term of the
    exact product of the float32 operands."""
    import torch
    rng = np.random.default_rng(11)
    M, N, K = 256, 256, 512
    a = rng.standard_normal((M, K)).astype(np.float32)
    b = rng.standard_normal((N, K)).astype(np.float32)
    at = torch.from_numpy(a).cuda(); bt = torch.from_numpy(b).cuda()
    ah = at.to(torch.bfloat16); al = (at - ah.float()).to(torch.bfloat16)
    bh = bt.to(torch.bfloat16); bl = (bt - bh.float()).to(torch.bfloat16)
    d, e = run_gemm(F, ah, al, bh, bl, 3)
    assert e == 0
    exact = a.astype(np.float64) @ b.astype(np.float64).T
    scale = np.abs(a).astype(np.float64) @ np.abs(b).astype(np.float64).T
    # per product: |x - hi - lo| <= 2^-16 |x| for both operands and the
    # dropped lo*lo <= 2^-16 |x y|; float32 accumulation <= K 2^-24 sum |xy|
    bound = (3 * 2.0 ** -16 + K * 2.0 ** -24) * scale
    assert np.all(np.abs(d - exact) <= bound)
    # and the typical error is far below the bound (random signs)
    assert rel(d, exact) < 2e-5


def test_gemm_wait_expires_without_loads(F):
    """A launch that issues no operand loads: the MMA issuer's bounded wait
    expires after about a second, the kernel sets the error word, stores
    nothing, frees its tensor memory and returns; the context stays usable."""
    rng = np.random.default_rng(5)
    a = bf16(rng.integers(-3, 4, (128, 128)))
    b = bf16(rng.integers(-3, 4, (128, 128)))
    d, e = run_gemm(F, a, a, b, b, 3, no_loads=1, fill=np.nan)
    assert e == 1
    assert np.all(np.isnan(d))
    d2, e2 = run_gemm(F, a, a, b, b, 1)
    assert e2 == 0
    ah = np.asarray(a.float().cpu().numpy(), np.float64)
    bh = np.asarray(b.float().cpu().numpy(), np.float64)
    assert np.array_equal(d2.astype(np.float64), ah @ bh.T)


def test_gemm_rejects_bad_shapes(F):
    import torch
    a = torch.zeros((128, 96), dtype=torch.bfloat16, device="cuda")
    d = torch.zeros((128, 128), dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(F.FFTPLError) as ei:
        F.fftpl_debug_tc_gemm(a, a, a, a, d, err)
    assert ei.value.status == F.FFTPL_EINVAL


# ------------------------------------------------------------- whole solve

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


def check_tc(got, ref):
    errs = {
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
    limits = {"rho": 1e-6, "psi": TOL_TC, "ex": TOL_TC, "ey": TOL_TC, "gN": TOL_TC,
              "gW": 1e-5, "N": TOL_TC, "hpwl": 1e-6, "tau": 1e-5}
    bad = {k: (errs[k], limits[k]) for k in errs if not errs[k] <= limits[k]}
    print("tensor-core path errors", {k: f"{v:.2e}" for k, v in errs.items()})
    assert not bad, f"parity failures {bad}; all {errs}"
    return errs


@pytest.mark.parametrize("name", ["medium", "precision_sub", "large"])
@pytest.mark.parametrize("det", [0, 1])
def test_tc_eval_parity(F, name, det):
    """n = 128 (one tile), 256 (the stage ring wraps) and 512 against the oracle."""
    inst = synth.make_instance(name)
    ref = oracle.eval_instance(inst, maps=True)
    got = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_BF16X3, deterministic=det)
    check_tc(got, ref)


def test_tc_deterministic_repeats_bitwise(F):
    inst = synth.make_instance("precision_sub")
    a = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_BF16X3, deterministic=1)
    b = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_BF16X3, deterministic=1)
    for k in ("psi", "ex", "ey", "gNx", "gNy"):
        assert np.array_equal(a[k], b[k]), k
    assert a["rep"]["N"] == b["rep"]["N"]


def oracle_samples(inst, count, seed):
    """psi, E_x, E_y of the oracle's series (Eqs. 9-12, FP64) at sampled bins
    of the instance's density map: (xs, ys, psi, ex, ey)."""
    n, m = inst.n, inst.m_mov
    fx = inst.fix_x if inst.m_fix else None
    fy = inst.fix_y if inst.m_fix else None
    fw = inst.w[m:] if inst.m_fix else None
    fh = inst.h[m:] if inst.m_fix else None
    rho, _, _ = oracle.density(inst.region, n, inst.target_density, inst.x, inst.y,
                               inst.w[:m], inst.h[:m], fx, fy, fw, fh)
    a = oracle.dct_coeffs(rho)
    rng = np.random.default_rng(seed)
    xs = rng.integers(0, n, count); ys = rng.integers(0, n, count)
    psi, ex, ey = oracle.potential_at(a, inst.region[2] - inst.region[0],
                                      inst.region[3] - inst.region[1], xs, ys)
    return xs, ys, psi, ex, ey


def test_tc_matches_fft_path_full_size(F):
    """At 2048 x 2048 bins (2.2M cells): psi, E_x, E_y at 64 sampled bins
    against the oracle's series, and every output against the transform
    path, within the tensor-core path's bound."""
    inst = synth.make_instance("precision")
    t = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_BF16X3)
    xs, ys, psi, ex, ey = oracle_samples(inst, 64, 2048)
    for k, ref in (("psi", psi), ("ex", ex), ("ey", ey)):
        assert rel(t[k][ys, xs], ref) < TOL_TC, k
    f = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_FFT)
    for k in ("psi", "ex", "ey"):
        assert rel(t[k], f[k]) < TOL_TC, k
    gt = np.concatenate([t["gNx"], t["gNy"]]); gf = np.concatenate([f["gNx"], f["gNy"]])
    assert rel(gt, gf) < TOL_TC
    assert abs(t["rep"]["N"] - f["rep"]["N"]) / abs(f["rep"]["N"]) < TOL_TC
    assert t["rep"]["tau"] == pytest.approx(f["rep"]["tau"], rel=1e-6)


def test_tc_in_the_loop(F):
    """The placement loop runs on the tensor-core path and follows the
    transform path's trajectory closely over the first iterations."""
    import torch
    inst = synth.make_instance("precision_sub")
    out = {}
    for path in (F.FFTPL_SOLVE_FFT, F.FFTPL_SOLVE_TC_BF16X3):
        with F.Problem(inst, solve_path=path, gamma_fixed=inst.gamma) as p:
            x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
            F.fftpl_place_init(p.h, x0, y0)
            recs, ran = F.fftpl_step(p.h, 10)
            assert ran == 10
            out[path] = recs
    a, b = out[F.FFTPL_SOLVE_FFT], out[F.FFTPL_SOLVE_TC_BF16X3]
    for k in ("hpwl", "N", "tau"):
        ra = np.array([r[k] for r in a]); rb = np.array([r[k] for r in b])
        assert np.allclose(ra, rb, rtol=1e-3, atol=1e-6), k


def test_tc_largest_grid_matches_fft_path(F):
    """n = 4096 (the largest grid, 600 MB of bf16 operands): 20000 random
    cells of a few bins each; the two solve paths agree within the
    tensor-core bound, and the energy is positive."""
    import synth as S
    rng = np.random.default_rng(4096)
    m = 20000
    L = 2048.0
    x, y, w, h = S.random_cells(rng, m, (0.0, 0.0, L, L), wmax=3.0, hmax=3.0)
    inst = S.make_instance("tiny")
    inst.n = 4096
    inst.region = (0.0, 0.0, L, L)
    inst.m_mov = m
    inst.m_fix = 0
    inst.w, inst.h, inst.x, inst.y = w, h, x, y
    inst.fix_x = np.zeros(0, np.float32); inst.fix_y = np.zeros(0, np.float32)
    inst.net_ptr = np.array([0, 2], np.int32); inst.pin_cell = np.array([0, 1], np.int32)
    inst.pin_dx = np.zeros(2, np.float32); inst.pin_dy = np.zeros(2, np.float32)
    t = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_TC_BF16X3)
    xs, ys, psi, ex, ey = oracle_samples(inst, 32, 4096)
    for k, ref in (("psi", psi), ("ex", ex), ("ey", ey)):
        assert rel(t[k][ys, xs], ref) < TOL_TC, k
    f = gpu_eval(F, inst, solve_path=F.FFTPL_SOLVE_FFT)
    for k in ("psi", "ex", "ey"):
        assert rel(t[k], f[k]) < TOL_TC, k
    assert rel(np.concatenate([t["gNx"], t["gNy"]]), np.concatenate([f["gNx"], f["gNy"]])) < TOL_TC
    assert t["rep"]["N"] == pytest.approx(f["rep"]["N"], rel=TOL_TC)
    assert t["rep"]["N"] > 0
