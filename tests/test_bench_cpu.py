"""The benchmark's FFT-based CPU comparator computes the same evaluation as
the oracle (its solve by library FFTs instead of explicit cosine sums), and
the per-step statistics helper reports what it says."""
import numpy as np
import pytest


@pytest.mark.parametrize("name", ["tiny", "medium"])
def test_cpu_fft_comparator_matches_oracle(orc, name):
    import bench
    import synth
    inst = synth.make_instance(name)
    ref = orc.eval_instance(inst, maps=True)
    got = bench.cpu_fft_eval(inst, {})
    for k in ("rho", "psi", "ex", "ey", "gNx", "gNy", "gWx", "gWy"):
        d = np.linalg.norm(np.ravel(got[k]) - np.ravel(ref[k])) / np.linalg.norm(np.ravel(ref[k]))
        assert d < 1e-12, k
    for k in ("N", "W", "hpwl", "tau"):
        assert got[k] == pytest.approx(ref[k], rel=1e-12), k


def test_step_stats():
    import bench
    st = bench.step_stats([float(v) for v in range(1, 101)])
    assert st["mean"] == 50.5 and st["median"] == 50.5 and st["count"] == 100
    assert st["p10"] == pytest.approx(10.9) and st["p90"] == pytest.approx(90.1)
