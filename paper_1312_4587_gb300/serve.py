"""Serving driver: a stream of placement jobs with Poisson arrivals fed to the
library's continuous-batching server (fftpl_server_*).

Jobs are synthetic instances (any object with the fields of a seeded
instance: region, n, w, h, m_mov, fix_x, fix_y, net_ptr, pin_cell, pin_dx,
pin_dy, x, y, target_density, gamma).  The driver submits each job when its
arrival time has passed on the wall clock, ticks the server in between, and
returns the server's statistics (jobs/s, per-iteration and per-job latency
percentiles).
"""
from __future__ import annotations

import time

import numpy as np

from . import fftpl as F


class Server:
    def __init__(self, budget_bytes=150 << 30, max_active=64, iters_per_tick=1,
                 deterministic=False, dry_run=False, workers=4):
        self.options = F.fftpl_server_default_options(
            hbm_budget_bytes=int(budget_bytes), max_active=int(max_active),
            iters_per_tick=int(iters_per_tick), deterministic=int(bool(deterministic)),
            dry_run=int(bool(dry_run)), workers=int(workers))
        self.s = F.fftpl_server_create(self.options)
        self.m = {}

    def submit(self, inst, iters, **opts):
        o = F.fftpl_default_options(target_density=float(getattr(inst, "target_density", 1.0)),
                                    gamma_fixed=float(getattr(inst, "gamma", 0.0)))
        for k, v in opts.items():
            setattr(o, k, v)
        jid = F.fftpl_server_submit(self.s, inst.region, inst.n, inst.w, inst.h, inst.m_mov,
                                    inst.fix_x, inst.fix_y, inst.net_ptr, inst.pin_cell,
                                    inst.pin_dx, inst.pin_dy, inst.x, inst.y, iters, o)
        self.m[jid] = inst.m_mov
        return jid

    def tick(self):
        return F.fftpl_server_tick(self.s)

    def drain(self, max_ticks=10**7):
        for _ in range(max_ticks):
            active, queued = self.tick()
            if active == 0 and queued == 0:
                return
        raise RuntimeError("server did not drain")

    def job(self, jid):
        return F.fftpl_server_job(self.s, jid, self.m.get(jid))

    def stats(self):
        return F.fftpl_server_report(self.s)

    def set_clock(self, now_s):
        F.fftpl_server_set_clock(self.s, now_s)

    def close(self):
        if self.s:
            F.fftpl_server_destroy(self.s)
            self.s = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def with_start(inst, seed):
    """The instance with its own seeded Gaussian start positions (a distinct
    placement job on the same netlist)."""
    import copy

    import synth
    j = copy.copy(inst)
    m = inst.m_mov
    j.x, j.y = synth.gaussian_start(np.random.default_rng(seed), inst.region, inst.w[:m],
                                    inst.h[:m])
    return j


def poisson_arrivals(rng, count, rate_per_s):
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))


def run_stream(jobs, arrivals, iters, server: Server, **opts):
    """Submits jobs[k] at wall time arrivals[k] (seconds from the start),
    ticking the server meanwhile; returns (stats, job ids)."""
    t0 = time.perf_counter()
    ids = []
    k = 0
    while k < len(jobs) or True:
        now = time.perf_counter() - t0
        while k < len(jobs) and arrivals[k] <= now:
            ids.append(server.submit(jobs[k], iters, **opts))
            k += 1
        active, queued = server.tick()
        if k >= len(jobs) and active == 0 and queued == 0:
            break
        if active == 0 and queued == 0 and k < len(jobs):
            time.sleep(max(0.0, min(0.01, arrivals[k] - (time.perf_counter() - t0))))
    return server.stats(), ids
