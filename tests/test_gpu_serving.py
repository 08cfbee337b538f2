"""Continuous batching on the GPU: a job's result is the same alone, in a mix
with jobs of other sizes and grid sizes running concurrently, and run
directly through fftpl_step (deterministic mode: bit-identical)."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1312_4587_gb300 import fftpl, serve
    fftpl.lib()
    return serve


def test_alone_equals_mix_equals_direct(S):
    import torch
    from paper_1312_4587_gb300 import fftpl as F
    a = synth.make_instance("tiny")
    others = [synth.make_instance("medium"), synth.make_instance("precision_sub")]
    iters = 40
    with S.Server(deterministic=True) as s:
        ja = s.submit(a, iters)
        s.drain()
        info, xa, ya = s.job(ja)
        assert info["state"] == F.FFTPL_JOB_DONE and info["iters_done"] == iters
    with S.Server(deterministic=True, max_active=8) as s:
        jb = s.submit(others[0], iters + 7)
        ja2 = s.submit(a, iters)
        jc = s.submit(others[1], iters - 9)
        s.drain()
        _, xm, ym = s.job(ja2)
        st = s.stats()
        # a shared the GPU with at least one other job (how many were active
        # at once depends on how fast the worker threads admit them)
        assert st["completed"] == 3 and st["peak_active"] >= 2
    assert np.array_equal(xa, xm) and np.array_equal(ya, ym)
    o = F.fftpl_default_options(target_density=a.target_density, gamma_fixed=a.gamma,
                                deterministic=1)
    with F.Problem(a, **{k: getattr(o, k) for k in ("target_density", "gamma_fixed", "deterministic")}) as p:
        x0 = torch.from_numpy(a.x).cuda(); y0 = torch.from_numpy(a.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        F.fftpl_step(p.h, iters)
        xd = torch.empty_like(x0); yd = torch.empty_like(y0)
        F.fftpl_place_positions(p.h, xd, yd)
    assert np.array_equal(xa, xd.cpu().numpy()) and np.array_equal(ya, yd.cpu().numpy())


def test_stream_of_jobs_completes(S):
    rng = np.random.default_rng(0)
    jobs = []
    for k in range(6):
        cfg = synth.serving_job_config(rng, m_lo=2000, m_hi=40000)
        jobs.append(synth.make_instance(cfg.name, seed=500 + k, cfg=cfg))
    arrivals = S.poisson_arrivals(rng, len(jobs), 200.0)
    with S.Server() as s:
        st, ids = S.run_stream(jobs, arrivals, 20, s)
        infos = [s.job(i)[0] for i in ids]
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert all(i["iters_done"] == 20 and i["hpwl"] > 0 for i in infos)
    assert st["iter_p99_ms"] >= st["iter_p50_ms"] > 0 and st["jobs_per_s"] > 0


def test_job_in_a_mix_matches_oracle(S):
    """A 10-iteration job served beside jobs of other sizes and grid sizes
    (float atomics, not the deterministic mode) follows the oracle's loop
    (Algorithm 1 with the Nesterov step) within the bounds of the direct
    loop's parity test: positions within 1e-4 relative L2, the last
    iteration's HPWL within 1e-4."""
    import oracle
    a = synth.make_instance("tiny")
    ox, oy, orows, oran = oracle.nesterov(a, 10, gamma_fixed=a.gamma)
    assert oran == 10
    with S.Server(max_active=8) as s:
        jb = s.submit(synth.make_instance("medium"), 25)
        ja = s.submit(a, 10)
        jc = s.submit(synth.make_instance("precision_sub"), 15)
        s.drain()
        info, xa, ya = s.job(ja)
        assert s.stats()["completed"] == 3
    assert info["iters_done"] == 10
    g = np.concatenate([xa, ya]).astype(np.float64)
    o = np.concatenate([ox, oy]).astype(np.float64)
    assert np.linalg.norm(g - o) / np.linalg.norm(o) < 1e-4
    assert abs(info["hpwl"] - orows[-1]["hpwl"]) <= 1e-4 * orows[-1]["hpwl"]
