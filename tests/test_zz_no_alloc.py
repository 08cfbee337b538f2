"""The allocation-free solve against the FP64 oracle and the regular density path.

fftpl_solve_noalloc serves callers that must not allocate device memory
while they run (host callbacks, services working from memory they set aside
up front, plugin hosts without an allocator).  It takes a density map and
caller-owned outputs, keeps its intermediates in a fixed array inside the
library, and must give the same potential and field as the handle-based
path and as the oracle's cosine series.  This file is named so that pytest
collects it last.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

TOL_MAP = 1e-5   # relative L2, as in the other parity tests
TOL_N = 2e-6


def rel(a, b):
    a = np.asarray(a, np.float64).ravel()
    b = np.asarray(b, np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


@pytest.fixture(scope="module")
def F():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1312_4587_gb300 import fftpl
    fftpl.lib()
    return fftpl


def outputs(n):
    import torch
    return [torch.full((n, n), np.nan, device="cuda") for _ in range(3)]


@pytest.mark.parametrize("name", ["medium", "precision_sub"])
def test_noalloc_matches_density_path(F, name):
    import torch
    inst = synth.make_instance(name)
    n = inst.n
    Lx = inst.region[2] - inst.region[0]
    Ly = inst.region[3] - inst.region[1]
    with F.Problem(inst) as p:
        x = torch.from_numpy(inst.x).cuda()
        y = torch.from_numpy(inst.y).cuda()
        N_ref = F.fftpl_density(p.h, x, y)
        f = F.fftpl_fields(p.h, n)
        rho = f["rho"].clone()
        ref = {k: f[k].cpu().numpy() for k in ("psi", "ex", "ey")}
    outs = outputs(n)
    torch.cuda.synchronize()
    free, used = [], []
    for call in range(3):
        N = F.fftpl_solve_noalloc(rho, n, Lx, Ly, *outs, want_N=True)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        used.append(torch.cuda.memory_allocated())
        got = dict(zip(("psi", "ex", "ey"), (t.cpu().numpy() for t in outs)))
        for k in ("psi", "ex", "ey"):
            assert rel(got[k], ref[k]) < TOL_MAP, (call, k, rel(got[k], ref[k]))
        assert abs(N - N_ref) / N_ref < TOL_N
        for t in outs:
            t.fill_(np.nan)
    # after the first call's set-up the calls take no device memory: torch's
    # own count is exact; the device-wide free memory (shared with other
    # processes) may only drift by a little
    assert used[1] == used[2]
    assert abs(free[1] - free[2]) <= 8 << 20


def test_noalloc_matches_oracle(F):
    """n = 128: the density of the 6001-cell instance, solved by the oracle's
    explicit cosine sums (Eqs. 9-12) in FP64, two calls in a row."""
    import torch
    inst = synth.make_instance("medium")
    n, m = inst.n, inst.m_mov
    Lx = inst.region[2] - inst.region[0]
    Ly = inst.region[3] - inst.region[1]
    rho, _, _ = oracle.density(inst.region, n, inst.target_density, inst.x, inst.y,
                               inst.w[:m], inst.h[:m], inst.fix_x, inst.fix_y,
                               inst.w[m:], inst.h[m:])
    _, psi, ex, ey = oracle.solve(rho, Lx, Ly)
    Nref = oracle.energy(rho, psi, (Lx / n) * (Ly / n))
    rd = torch.from_numpy(rho.astype(np.float32)).cuda()
    outs = outputs(n)
    for call in range(2):
        N = F.fftpl_solve_noalloc(rd, n, Lx, Ly, *outs, want_N=True)
        got = [t.cpu().numpy() for t in outs]
        for g, r in zip(got, (psi, ex, ey)):
            assert rel(g, r) < TOL_MAP, call
        assert abs(N - Nref) / Nref < TOL_N


def test_noalloc_largest_grid(F):
    """n = 1024, the largest grid (the whole scratch layout): a density made
    of three cosine modes has psi, E_x, E_y in closed form (Eqs. 11-12 for
    each mode); the constant part is dropped.  Run on a side stream without
    the energy read-back, twice."""
    import torch
    n, Lx, Ly = 1024, 1536.0, 768.0
    xs = (2 * np.arange(n) + 1) * np.pi / (2 * n)
    modes = [(1, 0, 0.7), (5, 9, -0.3), (300, 700, 0.05)]
    rho = np.full((n, n), 0.4)
    psi = np.zeros((n, n)); ex = np.zeros((n, n)); ey = np.zeros((n, n))
    for p, q, amp in modes:
        cx, sx = np.cos(p * xs), np.sin(p * xs)
        cy, sy = np.cos(q * xs), np.sin(q * xs)
        wp, wq = np.pi * p / Lx, np.pi * q / Ly
        d = wp * wp + wq * wq
        rho += amp * np.outer(cy, cx)
        psi += amp / d * np.outer(cy, cx)
        ex += amp * wp / d * np.outer(cy, sx)
        ey += amp * wq / d * np.outer(sy, cx)
    rd = torch.from_numpy(rho.astype(np.float32)).cuda()
    outs = outputs(n)
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    for call in range(2):
        with torch.cuda.stream(side):
            assert F.fftpl_solve_noalloc(rd, n, Lx, Ly, *outs, stream=side.cuda_stream) is None
        side.synchronize()
        got = [t.cpu().numpy() for t in outs]
        for g, r in zip(got, (psi, ex, ey)):
            assert rel(g, r) < TOL_MAP, call


def test_noalloc_rejects_bad_arguments(F):
    import torch
    big = torch.zeros(2048 * 2048 + 4, device="cuda")
    for n in (2048, 1000, 8, 0):
        with pytest.raises(F.FFTPLError) as ei:
            F.fftpl_solve_noalloc(big, n, 1.0, 1.0, big, big, big)
        assert ei.value.status == F.FFTPL_EINVAL
        assert "power of two" in str(ei.value)
    # a 4-byte offset view: the C ABI refuses it before any kernel runs
    n = 64
    with pytest.raises(F.FFTPLError) as ei:
        F.fftpl_solve_noalloc(big[1:], n, 1.0, 1.0, big, big, big)
    assert ei.value.status == F.FFTPL_EINVAL and "aligned" in str(ei.value)
    # the binding refuses wrong types and undersized outputs
    with pytest.raises(ValueError):
        F.fftpl_solve_noalloc(big[: n * n].double(), n, 1.0, 1.0, big, big, big)
    with pytest.raises(ValueError):
        F.fftpl_solve_noalloc(big, n, 1.0, 1.0, big[: n * n - 1], big, big)
    with pytest.raises(F.FFTPLError) as ei:
        F.fftpl_solve_noalloc(big, n, -1.0, 1.0, big, big, big)
    assert ei.value.status == F.FFTPL_EINVAL
