"""Benchmark: FFTPL objective-gradient evaluations per second on one GB300.

Workload (default): the precision instance -- 2.2M movable cells, 2.3M nets
(~8.15M pins), 150 macros covering 12 %, 2048 x 2048 bins -- seeded and
synthetic (it stands in for a BIGBLUE4-sized ISPD 2005 circuit).  One step =
one full objective-gradient evaluation: density scatter, spectral Poisson
solve (psi, E_x, E_y), field gather, WA wirelength and its gradient, and the
FP64 sums (N, W~, HPWL, tau, gradient norms).  Inputs are resident in HBM; L2
is flushed (256 MiB write) before every timed step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank evaluates its own replica
(weak scaling: no data-path collective; the problem does not shard).
--impl reference times the FP64 CPU oracle on the host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "gradient evals/s at 2M cells, 2048² bins; served jobs/s with p50/p99 latency"
UNIT = "evals/s"
WORKLOAD = "precision"

# algorithmic bytes per launch of each stage (float32 arrays read or written
# once; m movable cells, n bins per side, P pins, E nets)
def stage_bytes(m, n, P, E):
    nn = n * n
    return {
        "scatter": 16 * m + 8 * nn,           # x, y, w, h; zero + write D
        "rows_fwd": 12 * nn,                  # read D, M; write T1
        "cols": 12 * nn,                      # read T1; write PT, RT
        "rows_inv": 16 * nn,                  # read PT, RT; write E_x, E_y (psi on demand)
        "wa": 12 * P + 4 * E + 16 * m,        # pins, net_ptr, x, y; gradient out
        "cells": 16 * m + 8 * nn + 16 * m,    # x, y, w, h, E_x, E_y; read gW, write gN
    }


STAGE_IDS = {"scatter": 0, "rows_fwd": 1, "cols": 2, "rows_inv": 3, "wa": 4, "cells": 5}

# DRAM traffic per stage launch on the 2.2M-cell instance, dram__bytes_read.sum
# + dram__bytes_write.sum of the stage's kernels from one ncu --set full
# capture of this script (its summary is kept under profiles/), valid only
# while the kernel
# source it was taken from is unchanged: key = first 16 hex digits of the
# SHA-256 of the kernel file followed by fftpl_internal.cuh.
STAGE_TRAFFIC = {
    "scatter": ("k_density.cu", "fd2949651050cefb", 50778624 + 627968),
    "rows_fwd": ("k_spectral.cu", "a85e897b6059aa28", 33647616 + 16384),
    "cols": ("k_spectral.cu", "a85e897b6059aa28", 17206528 + 331520),
    "rows_inv": ("k_spectral.cu", "a85e897b6059aa28", 33614080 + 526336),
    # k_wa and k_wa_grp
    "wa": ("k_wire.cu", "a06baad7461894fc", 103047680 + 4505856 + 70472448 + 968704),
    "cells": ("k_wire.cu", "a06baad7461894fc", 76424960 + 14908672),
}


def source_key(fname):
    import hashlib
    h = hashlib.sha256()
    for p in (fname, "fftpl_internal.cuh"):
        with open(os.path.join(ROOT, "paper_1312_4587_gb300", "csrc", p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def stage_traffic(stage, workload):
    """ncu DRAM bytes per launch of a stage, or None if the kernel changed
    since the capture or the workload is another one."""
    if workload != "precision" or stage not in STAGE_TRAFFIC:
        return None
    fname, key, nbytes = STAGE_TRAFFIC[stage]
    return nbytes if source_key(fname) == key else None


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return 6800.0, 1900.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index=0):
        self.proc = None
        self.path = None
        self.index = index

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax = float(parts[2])
                except ValueError:
                    continue
                for nm, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value, ws):
    if ws <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def run_config(inst, args, ws):
    """The workload of a bench line (the same for both arms)."""
    m, n = inst.m_mov, inst.n
    E, P = inst.E, inst.P
    return {"workload": f"{inst.name}: {m} cells, {E} nets, {P} pins, {inst.m_fix} macros, "
                        f"{n}x{n} bins", "solve_path": "fft", "graphs": not args.no_graphs,
            "l2": "flushed before each timed step (256 MiB write)",
            "parallelism": f"replicas x{ws}"}


# ---------------------------------------------------------------- reference arm
def run_reference(args, ws, rank):
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import synth
    inst = synth.make_instance(WORKLOAD)
    oracle.build()
    cores = oracle.num_threads()
    times = []
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.eval_instance(inst)
        dt = time.perf_counter() - t0
        if k >= args.warmup:
            times.append(dt)
    tot = sum(times)
    val = args.steps / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": run_config(inst, args, ws),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "one full FP64 oracle evaluation of the same instance per step"},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_serving(args):
    """The serving workload: Poisson arrivals at
    50 jobs/s of 2,000 placement jobs with 5K-500K cells (log-uniform; bins
    the next power of two >= sqrt(cells), 12 % macros), 300 iterations each,
    under a 150 GB budget, with continuous batching.  The netlists come from a
    pool of distinct seeded instances and every job draws its own start
    positions.  Then the same jobs all at once (the server's capacity), and
    the first jobs of the stream one at a time for comparison."""
    import numpy as np

    import synth
    from paper_1312_4587_gb300 import serve

    rng = np.random.default_rng(1316)
    pool = []
    for k in range(args.serving_pool):
        cfg = synth.serving_job_config(rng)
        pool.append(synth.make_instance(cfg.name, seed=2000 + k, cfg=cfg))
    jobs = [serve.with_start(pool[k % len(pool)], 5000 + k) for k in range(args.serving_jobs)]
    arrivals = serve.poisson_arrivals(rng, len(jobs), args.serving_rate)
    cells = [j.m_mov for j in jobs]
    out = {"jobs": len(jobs), "distinct_netlists": len(pool),
           "start_positions": "one seeded Gaussian start per job",
           "arrival_rate_per_s": args.serving_rate, "iters_per_job": args.serving_iters,
           "budget_GB": 150, "cells": [int(min(cells)), int(max(cells))],
           "mean_cells": float(np.mean(cells))}

    def stats(st):
        return {"jobs_per_s": st["jobs_per_s"], "iter_p50_ms": st["iter_p50_ms"],
                "iter_p99_ms": st["iter_p99_ms"], "job_p50_ms": st["job_p50_ms"],
                "job_p99_ms": st["job_p99_ms"], "peak_active": st["peak_active"],
                "peak_device_GB": st["peak_device_bytes"] / 2**30,
                "completed": st["completed"], "failed": st["failed"]}

    with serve.Server(budget_bytes=150 << 30, max_active=64, iters_per_tick=5) as s:
        st, _ = serve.run_stream(jobs, arrivals, args.serving_iters, s)
    out.update(stats(st))
    # capacity: the same jobs all submitted at once, continuously batched
    with serve.Server(budget_bytes=150 << 30, max_active=64, iters_per_tick=5) as s:
        stc, _ = serve.run_stream(jobs, np.zeros(len(jobs)), args.serving_iters, s)
    out["saturated"] = stats(stc)
    # the first jobs of the stream one at a time, back to back
    k1 = min(len(jobs), args.serving_alone)
    with serve.Server(budget_bytes=150 << 30, max_active=1, iters_per_tick=5) as s:
        st1, _ = serve.run_stream(jobs[:k1], np.zeros(k1), args.serving_iters, s)
    out["alone"] = dict(stats(st1), jobs=k1)
    return out


def tc_flops(n):
    """FLOPs of one tensor-core solve: five products of 7 n^3 multiply-adds
    in total (G1, G2, G7: n^3 each; G35, G46: 2 n^3 each), three bf16
    products per multiply-add (hi*hi + hi*lo + lo*hi)."""
    return 2 * 3 * 7 * n ** 3


def tcr_flops(n):
    """FLOPs of one radix tensor-core solve: DFTs of 3 n rows in all (n/2 along
    x, n/2 + n along y, n along x back), each row 2 products of 2 x 128 x 128
    x n/64 multiply-adds, three bf16 products each."""
    return 3 * n * (2 * 2 * 128 * 128 * (n // 64)) * 3


def run_tc_path(args, inst, x, y, g, flush, stream, radix=False):
    """The same step on a tensor-core solve path (its own handle): the dense
    products (FFTPL_SOLVE_TC_BF16X3) or the radix DFTs (FFTPL_SOLVE_TC_RADIX);
    per-step time and the solve's stages against the bf16 peak."""
    import torch
    from paper_1312_4587_gb300 import fftpl as F
    path = F.FFTPL_SOLVE_TC_RADIX if radix else F.FFTPL_SOLVE_TC_BF16X3
    prob = F.Problem(inst, use_graphs=0 if args.no_graphs else 1, solve_path=path)
    h = prob.h
    for _ in range(max(3, args.warmup)):
        F.fftpl_eval(h, x, y, inst.gamma, *g, sync=False)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        F.fftpl_eval(h, x, y, inst.gamma, *g, sync=False)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    # the solve alone (density, solve and gather, no concurrent WA branch):
    # CUDA events around its three stages on the handle's stream
    F.fftpl_set_profiling(h, True)
    F.fftpl_stage_times(h, reset=True)
    for k in range(args.steps):
        flush.fill_(float(k))
        F.fftpl_density(h, x, y, g[0], g[1], sync=False)
    torch.cuda.synchronize()
    st, nl = F.fftpl_stage_times(h, reset=True)
    F.fftpl_check(h)
    prob.close()
    solve_ms = sum(st[i] / max(nl[i], 1) for i in (1, 2, 3))
    _, bf16, kind = load_peaks()
    flops = tcr_flops(inst.n) if radix else tc_flops(inst.n)
    tflops = flops / (solve_ms * 1e-3) / 1e12
    return {"solve_path": "tc_radix" if radix else "tc_bf16x3", "ms_per_step": round(ms, 5),
            "value": round(1000.0 / ms, 2), "unit": UNIT,
            "solve_ms": round(solve_ms, 5), "solve_flops": flops,
            "roofline": {"bound": "tensor", "achieved": round(tflops, 1),
                         "peak": bf16, "unit": "TFLOP/s",
                         "frac": round(tflops / bf16, 4),
                         "peak_kind": f"{kind} bf16 burst (solve timed alone)"}}


def run_variants(args, inst, x, y, g, flush, stream):
    """The same step with the model variants (each its own handle): the LSE
    wirelength and the Helmholtz smoothing of Eq. 4."""
    import math

    import torch
    from paper_1312_4587_gb300 import fftpl as F
    L = inst.region[2] - inst.region[0]
    out = {}
    for name, opts in (("lse", dict(wirelength=F.FFTPL_WL_LSE)),
                       ("helmholtz", dict(helmholtz_eps=4.0 * (math.pi / L) ** 2))):
        prob = F.Problem(inst, use_graphs=0 if args.no_graphs else 1, **opts)
        for _ in range(max(3, args.warmup)):
            F.fftpl_eval(prob.h, x, y, inst.gamma, *g, sync=False)
        torch.cuda.synchronize()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        for k in range(args.steps):
            flush.fill_(float(k))
            evs[k][0].record(stream)
            F.fftpl_eval(prob.h, x, y, inst.gamma, *g, sync=False)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
        F.fftpl_check(prob.h)
        prob.close()
        ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
        out[name] = {"value": round(1000.0 / ms, 2), "unit": UNIT, "ms_per_step": round(ms, 5),
                     "options": {k: (round(v, 9) if isinstance(v, float) else v)
                                 for k, v in opts.items()}}
    return out


def run_optimizers(args, x_inst):
    """Convergence of the two loop steps (Nesterov, and Algorithm 1's CG) on
    the 210K-cell and 2.2M-cell instances: iterations to tau <= 0.1 (at most
    1000), final HPWL, and time per iteration."""
    import time as _time

    import torch

    import synth
    from paper_1312_4587_gb300 import fftpl as F
    out = {}
    for inst in (synth.make_instance("large"), x_inst):
        x0 = torch.from_numpy(inst.x).cuda()
        y0 = torch.from_numpy(inst.y).cuda()
        res = {}
        for name, opt in (("nesterov", F.FFTPL_OPT_NESTEROV), ("cg", F.FFTPL_OPT_CG)):
            with F.Problem(inst, optimizer=opt, stop_on_tau=1) as p:
                F.fftpl_place_init(p.h, x0, y0)
                torch.cuda.synchronize()
                t0 = _time.perf_counter()
                rows, ran = F.fftpl_step(p.h, 1000)
                dt = _time.perf_counter() - t0
                F.fftpl_check(p.h)
            res[name] = {"iterations": ran, "tau": round(rows[-1]["tau"], 4),
                         "hpwl": round(rows[-1]["hpwl"], 1), "seconds": round(dt, 4),
                         "ms_per_iteration": round(1000.0 * dt / max(ran, 1), 4)}
        out[inst.name] = res
    return out


def run_fillers(args, inst, flush, stream):
    """The same step on the instance extended by the filler rule's cells
    (Section III-B): the cost of the extra pin-less movable cells."""
    import torch

    import synth
    from paper_1312_4587_gb300 import fftpl as F
    cnt, fw, fh = F.fftpl_fillers(inst.region, inst.w, inst.h, inst.m_mov, inst.fix_x,
                                  inst.fix_y, inst.target_density)
    ext = synth.with_fillers(inst, cnt, fw, fh)
    x = torch.from_numpy(ext.x).cuda()
    y = torch.from_numpy(ext.y).cuda()
    g = [torch.empty_like(x) for _ in range(4)]
    prob = F.Problem(ext, use_graphs=0 if args.no_graphs else 1)
    for _ in range(max(3, args.warmup)):
        F.fftpl_eval(prob.h, x, y, ext.gamma, *g, sync=False)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        F.fftpl_eval(prob.h, x, y, ext.gamma, *g, sync=False)
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    F.fftpl_check(prob.h)
    prob.close()
    ms = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    return {"fillers": cnt, "filler_size": [fw, fh], "cells": ext.m_mov,
            "value": round(1000.0 / ms, 2), "unit": UNIT, "ms_per_step": round(ms, 5)}


def step_stats(step_ms):
    """Mean, median and 10th/90th percentiles of per-step CUDA-event times."""
    import numpy as np
    a = np.asarray(step_ms, np.float64)
    return {"mean": round(float(a.mean()), 5), "median": round(float(np.median(a)), 5),
            "p10": round(float(np.percentile(a, 10)), 5),
            "p90": round(float(np.percentile(a, 90)), 5), "count": int(a.size)}


# ------------------------------------------------------- fast CPU comparator
def cpu_fft_eval(inst, cache):
    """One objective-gradient evaluation in FP64 on the host with the
    oracle's O(m) steps (exact overlaps, gather, WA) and the spectral solve
    of Eqs. 9-12 by library FFTs (scipy.fft / pocketfft, all cores: DCT-II
    forward, DCT-III and DST-III sums back) in place of the oracle's O(n^3)
    cosine sums: the fast CPU comparator of the timing table."""
    import numpy as np
    import scipy.fft as sf

    import oracle
    n, m = inst.n, inst.m_mov
    x0, y0, x1, y1 = inst.region
    Ab = ((x1 - x0) / n) * ((y1 - y0) / n)
    if "div" not in cache:
        u = np.arange(n)
        wu, wv = np.pi * u / (x1 - x0), np.pi * u / (y1 - y0)
        eps = np.where(u == 0, 1.0, 2.0)
        W2 = wv[:, None] ** 2 + wu[None, :] ** 2
        W2[0, 0] = np.inf
        # a = eps_u eps_v / n^2 sum rho cos cos (Eq. 10); scipy's DCT-II carries 2 per axis
        cache["div"] = (eps[:, None] * eps[None, :]) / (4.0 * n * n) / W2
        cache["wu"], cache["wv"] = wu, wv
    k = inst.m_fix
    fx, fy = (inst.fix_x, inst.fix_y) if k else (None, None)
    fw, fh = (inst.w[m:], inst.h[m:]) if k else (None, None)
    rho, D, Fm = oracle.density(inst.region, n, inst.target_density, inst.x, inst.y,
                                inst.w[:m], inst.h[:m], fx, fy, fw, fh)
    psi_hat = sf.dctn(rho, type=2, workers=-1) * cache["div"]

    def cos_sum(c, axis):        # sum_u c_u cos(pi u (2x+1) / 2n) along axis
        c = c.copy()
        sl = [slice(None)] * 2; sl[axis] = slice(1, None)
        c[tuple(sl)] *= 0.5
        return sf.dct(c, type=3, axis=axis, workers=-1)

    def sin_sum(c, axis):        # sum_{u>=1} c_u sin(pi u (2x+1) / 2n) along axis
        z = np.zeros_like(c)
        src = [slice(None)] * 2; dst = [slice(None)] * 2
        src[axis] = slice(1, None); dst[axis] = slice(0, n - 1)
        z[tuple(dst)] = 0.5 * c[tuple(src)]
        return sf.dst(z, type=3, axis=axis, workers=-1)

    cy = cos_sum(psi_hat, 0)
    psi = cos_sum(cy, 1)
    ex = sin_sum(cy * cache["wu"][None, :], 1)
    ey = cos_sum(sin_sum(psi_hat * cache["wv"][:, None], 0), 1)
    gNx, gNy = oracle.gather(inst.region, n, inst.x, inst.y, inst.w[:m], inst.h[:m], ex, ey)
    wa = oracle.wa(inst.net_ptr, inst.pin_cell, inst.pin_dx, inst.pin_dy, m, inst.x, inst.y,
                   inst.gamma, fx, fy)
    area = float(np.sum(inst.w[:m].astype(np.float64) * inst.h[:m].astype(np.float64)))
    return {"N": oracle.energy(rho, psi, Ab), "W": wa["W"], "hpwl": wa["hpwl"],
            "tau": oracle.overflow(D, Fm, Ab, inst.target_density, area),
            "gNx": gNx, "gNy": gNy, "gWx": wa["gcx"], "gWy": wa["gcy"],
            "psi": psi, "ex": ex, "ey": ey, "rho": rho}


def cpu_baselines(inst):
    """CPU timings beside the GPU line: the oracle on all host cores (the
    main cpu_baseline), the FFT-based FP64 comparator on all cores, and the
    oracle on one core (the paper's single-thread regime) on the 210K-cell
    512 x 512 instance (a full 2048 x 2048 evaluation on one core would take
    about a minute)."""
    import oracle
    import synth
    oracle.build()
    out = []
    cores = oracle.num_threads()
    t0 = time.perf_counter()
    oracle.eval_instance(inst)
    dt = time.perf_counter() - t0
    out.append({"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
                "sample": f"one full FP64 evaluation of the same instance ({dt:.1f} s)"})
    cache = {}
    cpu_fft_eval(inst, cache)
    reps = []
    for _ in range(3):
        t0 = time.perf_counter()
        cpu_fft_eval(inst, cache)
        reps.append(time.perf_counter() - t0)
    dt = statistics.median(reps)
    out.append({"value": 1.0 / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle_with_scipy_fft",
                "sample": f"median of 3 FP64 evaluations of the same instance, the oracle's "
                          f"solve replaced by scipy FFTs ({dt:.2f} s each)"})
    large = synth.make_instance("large")
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        oracle.eval_instance(large)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(cores)
    out.append({"value": 1.0 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"one FP64 oracle evaluation of the 210K-cell, 512 x 512 instance on one "
                          f"core ({dt:.1f} s); a different workload from the GPU line"})
    return out


def run_errors(args):
    """Relative L2 errors against the FP64 oracle on the 256 x 256 sub-problem
    of the precision instance (34K cells): every output of one evaluation on
    the transform and tensor-core solve paths, and the positions after 10
    placement iterations run directly and served in a mix of jobs."""
    import numpy as np
    import torch

    import oracle
    import synth
    from paper_1312_4587_gb300 import fftpl as F
    from paper_1312_4587_gb300 import serve

    def rel(a, b):
        a = np.asarray(a, np.float64).ravel(); b = np.asarray(b, np.float64).ravel()
        return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))

    inst = synth.make_instance("precision_sub")
    ref = oracle.eval_instance(inst, maps=True)
    out = {"workload": f"{inst.name}: {inst.m_mov} cells, {inst.n}x{inst.n} bins",
           "metric": "relative L2 vs FP64 oracle"}
    for name, path in (("fft_fp32", F.FFTPL_SOLVE_FFT), ("tc_bf16x3", F.FFTPL_SOLVE_TC_BF16X3)):
        with F.Problem(inst, solve_path=path) as p:
            xd = torch.from_numpy(inst.x).cuda(); yd = torch.from_numpy(inst.y).cuda()
            g = [torch.empty_like(xd) for _ in range(4)]
            rep = F.fftpl_eval(p.h, xd, yd, inst.gamma, *g)
            fl = F.fftpl_fields(p.h, inst.n)
            gg = [t.cpu().numpy() for t in g]
            out[name] = {
                "rho": rel(fl["rho"].cpu().numpy(), ref["rho"]),
                "psi": rel(fl["psi"].cpu().numpy(), ref["psi"]),
                "ex": rel(fl["ex"].cpu().numpy(), ref["ex"]),
                "ey": rel(fl["ey"].cpu().numpy(), ref["ey"]),
                "gradN": rel(np.concatenate(gg[:2]), np.concatenate([ref["gNx"], ref["gNy"]])),
                "gradW": rel(np.concatenate(gg[2:]), np.concatenate([ref["gWx"], ref["gWy"]])),
                "N": abs(rep["N"] - ref["N"]) / abs(ref["N"]),
                "W": abs(rep["W"] - ref["W"]) / abs(ref["W"]),
            }
    iters = 10
    ox, oy, _, _ = oracle.nesterov(inst, iters, gamma_fixed=inst.gamma)
    o = np.concatenate([ox, oy])
    with F.Problem(inst, gamma_fixed=inst.gamma) as p:
        x0 = torch.from_numpy(inst.x).cuda(); y0 = torch.from_numpy(inst.y).cuda()
        F.fftpl_place_init(p.h, x0, y0)
        F.fftpl_step(p.h, iters)
        xx = torch.empty_like(x0); yy = torch.empty_like(y0)
        F.fftpl_place_positions(p.h, xx, yy)
        direct = np.concatenate([xx.cpu().numpy(), yy.cpu().numpy()])
    with serve.Server(max_active=8) as s:
        s.submit(synth.make_instance("medium"), iters + 15)
        j = s.submit(inst, iters)
        s.submit(synth.make_instance("large"), iters + 5)
        s.drain()
        _, sx, sy = s.job(j)
    out["loop_positions_10_iters"] = {"direct_fp32": rel(direct, o),
                                      "served_in_mix_fp32": rel(np.concatenate([sx, sy]), o)}
    return out


# ---------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    import synth
    from paper_1312_4587_gb300 import fftpl as F

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    inst = synth.make_instance(args.workload)
    m, n, P, E = inst.m_mov, inst.n, inst.P, inst.E
    prob = F.Problem(inst, use_graphs=0 if args.no_graphs else 1)
    h = prob.h
    x = torch.from_numpy(inst.x).to(dev)
    y = torch.from_numpy(inst.y).to(dev)
    g = [torch.empty_like(x) for _ in range(4)]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        F.fftpl_eval(h, x, y, inst.gamma, *g, sync=False)

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    rep = F.fftpl_report(h)

    clocks = Clocks(local)
    clocks.start()
    barrier(ws)
    torch.cuda.synchronize()
    launches0 = F.fftpl_launch_count(h)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_wall = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(float(k))
        evs[k][0].record(stream)
        step()
        evs[k][1].record(stream)
    torch.cuda.synchronize()
    barrier(ws)
    t_wall = time.perf_counter() - t_wall
    launches = F.fftpl_launch_count(h) - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    ms_total = sum(step_ms)
    ms_max = max_over_ranks(ms_total, ws)
    clk = clocks.stop()

    # per-stage times (CUDA events on each stage's own stream), same steps
    F.fftpl_set_profiling(h, True)
    F.fftpl_stage_times(h, reset=True)
    for k in range(args.steps):
        flush.fill_(float(k))
        step()
    torch.cuda.synchronize()
    ms, nl = F.fftpl_stage_times(h, reset=True)
    F.fftpl_set_profiling(h, False)
    sb = stage_bytes(m, n, P, E)
    hbm, bf16, peak_kind = load_peaks()
    stages = {}
    for name, sid in STAGE_IDS.items():
        if nl[sid] == 0:
            continue
        per = ms[sid] / nl[sid]
        gbs = sb[name] / (per * 1e-3) / 1e9
        stages[name] = {"ms": round(per, 5), "GB/s": round(gbs, 1), "frac": round(gbs / hbm, 4),
                        "bytes": sb[name]}
    dom = max(stages, key=lambda k: stages[k]["ms"]) if stages else None

    # end to end through the C ABI with host buffers (pinned)
    hx = torch.from_numpy(inst.x).pin_memory()
    hy = torch.from_numpy(inst.y).pin_memory()
    hg = [torch.empty(m, dtype=torch.float32).pin_memory() for _ in range(4)]
    F.fftpl_eval_host(h, hx, hy, inst.gamma, *hg)
    barrier(ws)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        F.fftpl_eval_host(h, hx, hy, inst.gamma, *hg)
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(time.perf_counter() - t0, ws)

    value = ws * args.steps / (ms_max * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": run_config(inst, args, ws),
        "gpu_launches": int(launches),
        "step_ms": step_stats(step_ms),
        "e2e": {"value": ws * args.steps / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 8 * m,
                "d2h_bytes_per_step": 16 * m + 64},
        "clocks": clk,
        "stages": stages,
        "report": {k: rep[k] for k in ("N", "W", "hpwl", "tau")},
    }
    if dom:
        st = stages[dom]
        line["roofline"] = {"kernel": dom, "bound": "hbm", "achieved": st["GB/s"], "peak": hbm,
                            "unit": "GB/s", "frac": st["frac"],
                            "traffic": stage_traffic(dom, args.workload),
                            "algorithmic_bytes": st["bytes"], "peak_kind": peak_kind}
    if rank == 0 and ws == 1 and not args.no_optimizers:
        line["optimizers"] = run_optimizers(args, inst)
    if not args.no_variants:
        line["variants"] = run_variants(args, inst, x, y, g, flush, stream)
        line["variants"]["fillers"] = run_fillers(args, inst, flush, stream)
    if not args.no_tc_path and n >= F.FFTPL_TC_MIN_N:
        line["tc_path"] = run_tc_path(args, inst, x, y, g, flush, stream)
    if not args.no_tc_path and n >= F.FFTPL_TCR_MIN_N:
        line["tc_radix_path"] = run_tc_path(args, inst, x, y, g, flush, stream, radix=True)
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cb = cpu_baselines(inst)
        line["cpu_baseline"] = cb[0]
        line["cpu_baselines"] = cb
    if rank == 0 and ws == 1 and not args.no_errors:
        line["errors"] = run_errors(args)
    if rank == 0 and ws == 1 and args.serving_jobs > 0:
        line["serving"] = run_serving(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    prob.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-graphs", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-optimizers", action="store_true",
                    help="skip the Nesterov / CG convergence comparison")
    ap.add_argument("--no-variants", action="store_true",
                    help="skip the LSE / Helmholtz variant timings")
    ap.add_argument("--no-errors", action="store_true",
                    help="skip the per-result errors against the oracle")
    ap.add_argument("--no-tc-path", action="store_true",
                    help="skip the tensor-core solve path comparison")
    ap.add_argument("--serving-jobs", type=int, default=2000,
                    help="jobs in the serving stream (0: skip)")
    ap.add_argument("--serving-pool", type=int, default=64,
                    help="distinct netlists the stream's jobs draw from")
    ap.add_argument("--serving-alone", type=int, default=200,
                    help="jobs of the stream also run one at a time")
    ap.add_argument("--serving-rate", type=float, default=50.0)
    ap.add_argument("--serving-iters", type=int, default=300)
    args = ap.parse_args()
    ws, rank, local = dist_env()
    if ws > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if (args.impl == "ours" and torch.cuda.is_available()) else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    try:
        if args.impl == "reference":
            return run_reference(args, ws, rank)
        return run_ours(args, ws, rank, local)
    finally:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    sys.exit(main())
