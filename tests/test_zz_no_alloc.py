"""The allocation-free solve against the regular density path.

fftpl_solve_noalloc serves callers that must not allocate device memory
while they run (host callbacks, services working from memory they set aside
up front, plugin hosts without an allocator).  It takes a density map and
caller-owned outputs, keeps its intermediates in a fixed array inside the
library, and must give the same potential and field as the handle-based
path.  This file is named so that pytest collects it last.
"""
import numpy as np
import pytest

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
    outs = [torch.full((n, n), np.nan, device="cuda") for _ in range(3)]
    free = []
    for call in range(3):
        N = F.fftpl_solve_noalloc(rho, n, Lx, Ly, *outs, want_N=True)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = dict(zip(("psi", "ex", "ey"), (t.cpu().numpy() for t in outs)))
        for k in ("psi", "ex", "ey"):
            assert rel(got[k], ref[k]) < TOL_MAP, (call, k, rel(got[k], ref[k]))
        assert abs(N - N_ref) / N_ref < TOL_N
        for t in outs:
            t.fill_(np.nan)
    # after the first call's set-up, calls leave free device memory unchanged
    assert free[1] == free[2]


def test_noalloc_rejects_oversize_grid(F):
    import torch
    n = 2048
    rho = torch.zeros(16, device="cuda")
    with pytest.raises(F.FFTPLError) as ei:
        F.fftpl_solve_noalloc(rho, n, 1.0, 1.0, rho, rho, rho)
    assert ei.value.status == F.FFTPL_EINVAL
    assert "1024" in str(ei.value)
