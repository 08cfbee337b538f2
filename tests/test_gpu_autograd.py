"""DensityEnergy (torch.autograd.Function): forward = scatter + spectral
solve, backward = the field-gather kernel (or the exact adjoint), on the
differentiation instance (500K cells, 1024x1024 bins).

Central finite differences of the binned energy are computed in FP64 from
the oracle: N is a quadratic form 1/2 A_b rho^T G rho with G symmetric, so
for a step +-h that moves no cell edge across a bin edge,
  N(x+h) - N(x-h) = A_b psi . (rho(x+h) - rho(x-h))
exactly (the quadratic terms cancel), which needs only the oracle's psi and
the moved cell's own overlap map.
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


@pytest.fixture(scope="module")
def diff_case():
    inst = synth.make_instance("diff")
    ref = oracle.eval_instance(inst, maps=True)
    return inst, ref


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def test_backward_is_the_gather(F, diff_case):
    import torch
    from paper_1312_4587_gb300.autograd import density_energy
    inst, ref = diff_case
    with F.Problem(inst) as p:
        x = torch.from_numpy(inst.x).cuda().requires_grad_(True)
        y = torch.from_numpy(inst.y).cuda().requires_grad_(True)
        N = density_energy(x, y, p, "gather")
        (2.5 * N).backward()
        assert abs(N.item() - ref["N"]) / ref["N"] < 2e-6
        gx = x.grad.cpu().numpy() / 2.5
        gy = y.grad.cpu().numpy() / 2.5
    assert rel(np.concatenate([gx, gy]), np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5


def test_adjoint_against_central_differences(F, diff_case):
    import torch
    from paper_1312_4587_gb300.autograd import density_energy
    inst, ref = diff_case
    m = inst.m_mov
    wb = inst.wb
    h = 1e-3 * wb
    rng = np.random.default_rng(3)
    edges = lambda c, s: (np.float32(c) - np.float32(0.5) * np.float32(s),
                          np.float32(c) + np.float32(0.5) * np.float32(s))
    cells = []
    for i in rng.permutation(m):
        ok = True
        for c, s, e0 in ((inst.x[i], inst.w[i], inst.region[0]), (inst.y[i], inst.h[i], inst.region[1])):
            for e in edges(c, s):
                r = (float(e) - e0) / wb
                if abs(r - round(r)) * wb < 4 * h or float(e) <= e0 or float(e) >= e0 + inst.n * wb:
                    ok = False
        if ok:
            cells.append(i)
        if len(cells) == 64:
            break
    cells = np.array(cells)
    psi = ref["psi"]
    fd = []
    for i in cells:
        row = []
        for axis in (0, 1):
            xs = np.array([inst.x[i]] * 2, np.float32)
            ys = np.array([inst.y[i]] * 2, np.float32)
            step = np.float32(h)
            if axis == 0:
                xs[0] += step; xs[1] -= step
            else:
                ys[0] += step; ys[1] -= step
            dp = float(xs[0] - inst.x[i]) if axis == 0 else float(ys[0] - inst.y[i])
            dm = float(inst.x[i] - xs[1]) if axis == 0 else float(inst.y[i] - ys[1])
            op = oracle.overlap_map(inst.region, inst.n, xs[:1], ys[:1], inst.w[i:i + 1], inst.h[i:i + 1])
            om = oracle.overlap_map(inst.region, inst.n, xs[1:], ys[1:], inst.w[i:i + 1], inst.h[i:i + 1])
            row.append(float(np.sum(psi * (op - om))) / (dp + dm))
        fd.append(row)
    fd = np.array(fd)
    ax, ay = oracle.adjoint(inst.region, inst.n, inst.x[cells], inst.y[cells], inst.w[cells],
                            inst.h[cells], psi)
    # the oracle's adjoint is the exact derivative
    assert rel(np.stack([ax, ay], 1), fd) < 1e-9
    with F.Problem(inst) as p:
        x = torch.from_numpy(inst.x).cuda().requires_grad_(True)
        y = torch.from_numpy(inst.y).cuda().requires_grad_(True)
        density_energy(x, y, p, "adjoint").backward()
        g = np.stack([x.grad.cpu().numpy()[cells], y.grad.cpu().numpy()[cells]], 1)
    err = rel(g, fd)
    # psi carries ~2e-7 relative error; the adjoint differences psi between the
    # bins holding a cell's two edges, which cancels part of it
    assert err < 1e-4, err
    # the paper's gather is a different (smoothed) derivative; report the gap
    gap = rel(np.stack([ref["gNx"][cells], ref["gNy"][cells]], 1), fd)
    print(f"adjoint vs FD {err:.2e}; gather vs FD {gap:.2e}")


def test_stale_maps_are_recomputed(F):
    import torch
    from paper_1312_4587_gb300.autograd import density_energy
    inst = synth.make_instance("medium")
    ref = oracle.eval_instance(inst)
    with F.Problem(inst) as p:
        x = torch.from_numpy(inst.x).cuda().requires_grad_(True)
        y = torch.from_numpy(inst.y).cuda().requires_grad_(True)
        N1 = density_energy(x, y, p)
        # a second forward at other positions overwrites the handle's maps
        density_energy(x.detach() + 1.0, y.detach(), p)
        N1.backward()
        g = np.concatenate([x.grad.cpu().numpy(), y.grad.cpu().numpy()])
    assert rel(g, np.concatenate([ref["gNx"], ref["gNy"]])) < 1e-5
