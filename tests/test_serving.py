"""Serving scheduler bookkeeping on the host (dry runs: no device work):
admission never exceeds the HBM budget, jobs are admitted in arrival order,
a job larger than the whole budget fails instead of blocking the queue, and
per-job / per-iteration latencies follow an injected clock."""
import numpy as np
import pytest

import synth


@pytest.fixture(scope="module")
def serve():
    from paper_1312_4587_gb300 import _build
    _build.build()
    from paper_1312_4587_gb300 import serve as S
    return S


def jobs_of_sizes(ms):
    out = []
    for k, m in enumerate(ms):
        cfg = synth.scaled_config("tiny", m, name=f"j{k}")
        out.append(synth.make_instance(cfg.name, seed=100 + k, cfg=cfg))
    return out


def test_budget_fifo_and_latency(serve):
    from paper_1312_4587_gb300 import fftpl as F
    jobs = jobs_of_sizes([1000, 4000, 1000, 16000, 2000, 1000])
    est = [F.fftpl_estimate_bytes(j.n, j.m_mov, j.m_fix, j.E, j.P, 5, 0) for j in jobs]
    budget = max(est) + min(est)        # room for the largest job plus the smallest
    with serve.Server(budget_bytes=budget, max_active=4, dry_run=True) as s:
        s.set_clock(0.0)
        ids = [s.submit(j, 5) for j in jobs]
        t = 0.0
        held_max = 0
        for tick in range(200):
            t += 0.010
            s.set_clock(t)
            active, queued = s.tick()
            held = sum(s.job(i)[0]["device_bytes"] for i in ids if s.job(i)[0]["state"] == 1)
            held_max = max(held_max, held)
            assert held <= budget
            if active == 0 and queued == 0:
                break
        st = s.stats()
        infos = [s.job(i)[0] for i in ids]
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["peak_device_bytes"] <= budget and held_max <= budget
    admits = [i["t_admit"] for i in infos]
    assert admits == sorted(admits)                      # arrival order
    for i in infos:
        assert i["iters_done"] == 5
        # one iteration per tick, the first in the admitting tick: done 4 ticks
        # (of 10 ms) after admission
        assert abs((i["t_done"] - i["t_admit"]) - 0.040) < 1e-9
    lat = sorted(1e3 * (i["t_done"] - i["t_submit"]) for i in infos)
    assert abs(st["job_p50_ms"] - np.percentile(lat, 50)) < 1e-6
    assert abs(st["job_p99_ms"] - np.percentile(lat, 99)) < 1e-6
    # a job's iterations complete one tick (10 ms) apart; its first one within
    # the admitting tick, which takes no time on the injected clock
    assert abs(st["iter_p50_ms"] - 10.0) < 1e-6 and abs(st["iter_p99_ms"] - 10.0) < 1e-6


def test_job_larger_than_budget_fails_not_blocks(serve):
    from paper_1312_4587_gb300 import fftpl as F
    small, big = jobs_of_sizes([1000, 60000])
    budget = F.fftpl_estimate_bytes(small.n, small.m_mov, small.m_fix, small.E, small.P, 3, 0) * 2
    with serve.Server(budget_bytes=budget, dry_run=True) as s:
        s.set_clock(0.0)
        jb = s.submit(big, 3)
        js = s.submit(small, 3)
        with pytest.raises(F.FFTPLError) as e:
            s.tick()
        assert e.value.status == F.FFTPL_ENOMEM
        s.drain()
        assert s.job(jb)[0]["state"] == F.FFTPL_JOB_FAILED
        assert s.job(js)[0]["state"] == F.FFTPL_JOB_DONE
        assert s.stats()["failed"] == 1


def test_iters_per_tick_and_slots(serve):
    jobs = jobs_of_sizes([1000] * 5)
    with serve.Server(max_active=2, iters_per_tick=3, dry_run=True) as s:
        s.set_clock(0.0)
        ids = [s.submit(j, 7) for j in jobs]
        peak = 0
        for t in range(1, 100):
            s.set_clock(t * 0.01)
            a, q = s.tick()
            peak = max(peak, a)
            if a == 0 and q == 0:
                break
        st = s.stats()
        infos = [s.job(i)[0] for i in ids]
    assert st["peak_active"] == 2 and st["completed"] == 5
    # 7 iterations at 3 per tick take 3 ticks: done 2 ticks after admission
    assert all(abs(i["t_done"] - i["t_admit"] - 0.02) < 1e-9 for i in infos)
    assert all(i["iters_done"] == 7 for i in infos)
