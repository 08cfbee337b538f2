"""The transform path's transposed stores through the TMA unit against plain
per-thread stores: the same values bit for bit (deterministic mode, so that
the density map itself is bit-identical between the two evaluations), at
grid sizes from the smallest box (n = 16) to the 256-row boxes."""
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


def instance(name):
    if name.startswith("tiny_n"):
        base = synth.make_instance("tiny")
        d = dict(base.__dict__)
        d["n"] = int(name[len("tiny_n"):])
        return synth.Instance(**d)
    return synth.make_instance(name)


@pytest.mark.parametrize("name", ["tiny_n16", "tiny_n64", "precision_sub", "large", "diff"])
def test_transpose_stores_bit_exact(F, name):
    import torch
    inst = instance(name)
    x = torch.from_numpy(np.ascontiguousarray(inst.x)).cuda()
    y = torch.from_numpy(np.ascontiguousarray(inst.y)).cuda()
    out = []
    with F.Problem(inst, deterministic=1) as p:
        for tma in (True, False, True):
            F.fftpl_debug_transpose_stores(p.h, tma)
            g = [torch.empty_like(x) for _ in range(4)]
            rep = F.fftpl_eval(p.h, x, y, inst.gamma, *g)
            fl = {k: v.cpu().numpy().copy() for k, v in F.fftpl_fields(p.h, inst.n).items()}
            F.fftpl_check(p.h)
            out.append((rep, fl, [t.cpu().numpy() for t in g]))
    (r0, f0, g0), (r1, f1, g1), (r2, f2, g2) = out
    for k in ("psi", "ex", "ey"):
        assert np.array_equal(f0[k], f1[k]), k
        assert np.array_equal(f0[k], f2[k]), k
    for a, b in zip(g0, g1):
        assert np.array_equal(a, b)
    assert r0["N"] == r1["N"] == r2["N"]
