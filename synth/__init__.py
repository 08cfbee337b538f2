"""Seeded synthetic placement instances.

This module only draws random netlists, cell sizes, macros and start positions.
It holds none of the placement method's arithmetic (no overlap areas, no
transforms, no wirelength), so both the FP64 oracle and the CUDA library can be
fed from it without sharing any computation.

The instances stand in for the ISPD 2005 circuits used in Table I of the FFTPL
paper (those files are not available here).  Their shape follows the paper's
problem statement (Section II: hypergraph G=(V,E,R), movable cells V_m, fixed
macros V_f, an n x n bin grid over R) and the workload recipe:

* cells are one row (1 unit) high; widths are lognormal with median 2 sites and
  sigma 0.6, rounded to whole sites, at least 1 and at most 40 (the tiny
  instance uses integer widths uniform in 1..4);
* nets: 60 % two-pin, 25 % three- or four-pin, 15 % with degree 5..50 drawn
  from p(d) ~ d^-2.5 (the tiny instance uses degrees uniform in 2..5); each net
  picks an anchor in a random permutation of the cells and draws its other
  pins without replacement from a +-64 window around it, so the netlist is
  local rather than an expander; about 1 % of nets also get a pin on a macro;
* pin offsets are uniform inside the cell (relative to the cell centre);
* fixed macros are non-overlapping rectangles with aspect ratio in [0.5, 2]
  covering a stated fraction of the region, with integer corners;
* start positions are Gaussian around the region centre, sigma = L/10 per
  axis, clamped so that each cell lies inside the region.

All coordinates and sizes are float32, indices int32.  Region corners and bin
widths are chosen so that every bin edge x0 + k*w_b is exact in float32.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

SEED_BASE = 1312


@dataclass(frozen=True)
class Config:
    name: str
    L: float            # region side (square region [0, L]^2)
    n: int              # bins per side
    m: int              # movable cells
    E: int              # nets
    n_macros: int
    macro_frac: float   # fraction of the region covered by macros
    target_density: float
    gamma_bins: float   # WA gamma in bin widths (used when fixed)
    tiny_widths: bool = False
    degree_uniform: tuple | None = None
    index: int = 0

    @property
    def wb(self) -> float:
        return self.L / self.n


CONFIGS = {
    # Plain method, tiny instance: 128x128 units, 64x64 bins, 1000 cells,
    # 1200 nets with degree uniform in 2..5, no macros, rho_t = 1.0.
    "tiny": Config("tiny", 128.0, 64, 1000, 1200, 0, 0.0, 1.0, 0.5,
                   tiny_widths=True, degree_uniform=(2, 5), index=0),
    # Large plain FP32 (ADAPTEC1-sized): 210K cells, 220K nets, 40 macros
    # covering 12 %, 512x512 bins, rho_t = 0.9.
    "large": Config("large", 1024.0, 512, 210_000, 220_000, 40, 0.12, 0.9, 0.5,
                    index=1),
    # Precision (BIGBLUE4-sized): 2.2M cells, 2.3M nets, 150 macros, 2048^2.
    "precision": Config("precision", 3072.0, 2048, 2_200_000, 2_300_000, 150,
                        0.12, 0.9, 0.5, index=2),
    # Differentiation: 500K cells, 1024^2 bins, no macros.
    "diff": Config("diff", 1536.0, 1024, 500_000, 524_000, 0, 0.0, 1.0, 0.5,
                   index=3),
    # The 256x256 sub-problem of the precision instance (same generator and
    # density, 1/64 of the cells and nets).
    "precision_sub": Config("precision_sub", 384.0, 256, 34_375, 35_937, 3,
                            0.12, 0.9, 0.5, index=2),
    # A mid-size instance spanning several tiles with a ragged tail; small
    # enough for the oracle's O(n^3) cosine sums to finish in seconds.
    "medium": Config("medium", 192.0, 128, 6_001, 6_301, 5, 0.12, 0.9, 0.5,
                     index=5),
}


@dataclass
class Instance:
    name: str
    region: tuple          # (x0, y0, x1, y1) float64, exact in float32
    n: int
    target_density: float
    gamma: float           # WA smoothing parameter in placement units
    m_mov: int
    m_fix: int
    w: np.ndarray          # float32 [m_mov + m_fix] (movable first)
    h: np.ndarray          # float32 [m_mov + m_fix]
    fix_x: np.ndarray      # float32 [m_fix] macro centres
    fix_y: np.ndarray
    net_ptr: np.ndarray    # int32 [E + 1]
    pin_cell: np.ndarray   # int32 [P]  (movable id, or m_mov + macro id)
    pin_dx: np.ndarray     # float32 [P] offset from the cell centre
    pin_dy: np.ndarray
    x: np.ndarray          # float32 [m_mov] start positions (centres)
    y: np.ndarray
    seed: int = 0
    extra: dict = field(default_factory=dict)

    @property
    def E(self) -> int:
        return int(self.net_ptr.shape[0] - 1)

    @property
    def P(self) -> int:
        return int(self.pin_cell.shape[0])

    @property
    def wb(self) -> float:
        return (self.region[2] - self.region[0]) / self.n

    @property
    def hb(self) -> float:
        return (self.region[3] - self.region[1]) / self.n


# ----------------------------------------------------------------------------
# pieces
# ----------------------------------------------------------------------------

def cell_widths(rng: np.random.Generator, m: int, tiny: bool = False) -> np.ndarray:
    if tiny:
        return rng.integers(1, 5, size=m).astype(np.float32)
    w = np.rint(np.exp(rng.normal(math.log(2.0), 0.6, size=m)))
    return np.clip(w, 1, 40).astype(np.float32)


def net_degrees(rng: np.random.Generator, E: int, uniform: tuple | None = None) -> np.ndarray:
    if uniform is not None:
        lo, hi = uniform
        return rng.integers(lo, hi + 1, size=E).astype(np.int64)
    kind = rng.random(E)
    deg = np.full(E, 2, dtype=np.int64)
    mid = (kind >= 0.60) & (kind < 0.85)
    deg[mid] = rng.integers(3, 5, size=int(mid.sum()))
    big = kind >= 0.85
    ds = np.arange(5, 51)
    p = ds.astype(np.float64) ** -2.5
    p /= p.sum()
    deg[big] = rng.choice(ds, size=int(big.sum()), p=p)
    return deg


def _distinct_offsets(rng: np.random.Generator, cnt: int, k: int, window: int = 64) -> np.ndarray:
    """cnt rows of k distinct nonzero offsets in [-window, window]."""
    span = 2 * window  # candidates 0..span-1 mapped to -window..-1, 1..window
    if k == 0:
        return np.zeros((cnt, 0), dtype=np.int64)
    if k <= 12:
        out = rng.integers(0, span, size=(cnt, k))
        while True:
            s = np.sort(out, axis=1)
            bad = np.any(s[:, 1:] == s[:, :-1], axis=1) if k > 1 else np.zeros(cnt, bool)
            nb = int(bad.sum())
            if nb == 0:
                break
            out[bad] = rng.integers(0, span, size=(nb, k))
    else:
        keys = rng.random((cnt, span))
        out = np.argsort(keys, axis=1)[:, :k]
    return np.where(out < window, out - window, out - window + 1)


def netlist(rng: np.random.Generator, m: int, E: int, w: np.ndarray, h: np.ndarray,
            uniform_degree: tuple | None = None, window: int = 64):
    deg = net_degrees(rng, E, uniform_degree)
    deg = np.minimum(deg, m)
    perm = rng.permutation(m)
    anchor = rng.integers(0, m, size=E)
    net_ptr = np.zeros(E + 1, dtype=np.int64)
    np.cumsum(deg, out=net_ptr[1:])
    P = int(net_ptr[-1])
    pin_cell = np.empty(P, dtype=np.int64)
    for d in np.unique(deg):
        idx = np.nonzero(deg == d)[0]
        k = int(d) - 1
        offs = _distinct_offsets(rng, idx.size, k, window=min(window, max(1, (m - 1) // 2)))
        cells = np.empty((idx.size, int(d)), dtype=np.int64)
        cells[:, 0] = perm[anchor[idx]]
        if k:
            cells[:, 1:] = perm[(anchor[idx, None] + offs) % m]
        starts = net_ptr[idx]
        pos = starts[:, None] + np.arange(int(d))[None, :]
        pin_cell[pos.ravel()] = cells.ravel()
    pc = pin_cell.astype(np.int64)
    dx = ((rng.random(P) - 0.5) * w[pc]).astype(np.float32)
    dy = ((rng.random(P) - 0.5) * h[pc]).astype(np.float32)
    return net_ptr.astype(np.int32), pin_cell.astype(np.int32), dx, dy


def macros(rng: np.random.Generator, L: float, count: int, frac: float, max_tries: int = 20000):
    """Non-overlapping macros with integer corners; returns (cx, cy, w, h)."""
    if count == 0 or frac <= 0:
        z = np.zeros(0, np.float32)
        return z, z, z, z
    target = frac * L * L
    areas = rng.uniform(0.5, 1.5, size=count)
    areas *= target / areas.sum()
    rects = []
    for a in areas:
        for _ in range(max_tries):
            asp = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
            mw = max(2.0, float(round(math.sqrt(a * asp))))
            mh = max(2.0, float(round(a / mw)))
            if mw >= L - 2 or mh >= L - 2:
                a *= 0.9
                continue
            lx = float(rng.integers(1, int(L - mw)))
            ly = float(rng.integers(1, int(L - mh)))
            ok = True
            for (ox, oy, ow, oh) in rects:
                if lx < ox + ow + 1 and ox < lx + mw + 1 and ly < oy + oh + 1 and oy < ly + mh + 1:
                    ok = False
                    break
            if ok:
                rects.append((lx, ly, mw, mh))
                break
            a *= 0.995
    r = np.array(rects, dtype=np.float64).reshape(-1, 4)
    cx = (r[:, 0] + 0.5 * r[:, 2]).astype(np.float32)
    cy = (r[:, 1] + 0.5 * r[:, 3]).astype(np.float32)
    return cx, cy, r[:, 2].astype(np.float32), r[:, 3].astype(np.float32)


def gaussian_start(rng: np.random.Generator, region, w: np.ndarray, h: np.ndarray,
                   sigma_frac: float = 0.1):
    x0, y0, x1, y1 = region
    m = w.shape[0]
    cx, cy = 0.5 * (x0 + x1), 0.5 * (y0 + y1)
    x = rng.normal(cx, sigma_frac * (x1 - x0), size=m)
    y = rng.normal(cy, sigma_frac * (y1 - y0), size=m)
    x = np.clip(x, x0 + 0.5 * w, x1 - 0.5 * w)
    y = np.clip(y, y0 + 0.5 * h, y1 - 0.5 * h)
    return x.astype(np.float32), y.astype(np.float32)


def _macro_pins(rng, net_ptr, pin_cell, dx, dy, m_mov, fw, fh, frac=0.01):
    """Move the last pin of about `frac` of the nets onto a random macro."""
    k = fw.shape[0]
    E = net_ptr.shape[0] - 1
    if k == 0 or E == 0:
        return
    sel = np.nonzero(rng.random(E) < frac)[0]
    last = net_ptr[sel + 1].astype(np.int64) - 1
    mid = rng.integers(0, k, size=sel.size)
    pin_cell[last] = (m_mov + mid).astype(np.int32)
    dx[last] = ((rng.random(sel.size) - 0.5) * fw[mid]).astype(np.float32)
    dy[last] = ((rng.random(sel.size) - 0.5) * fh[mid]).astype(np.float32)


# ----------------------------------------------------------------------------
# instances
# ----------------------------------------------------------------------------

def make_instance(name: str, seed: int | None = None, cfg: Config | None = None) -> Instance:
    cfg = cfg or CONFIGS[name]
    seed = SEED_BASE + cfg.index if seed is None else seed
    rng = np.random.Generator(np.random.PCG64(seed))
    L = cfg.L
    region = (0.0, 0.0, float(L), float(L))
    w_mov = cell_widths(rng, cfg.m, cfg.tiny_widths)
    h_mov = np.ones(cfg.m, dtype=np.float32)
    fx, fy, fw, fh = macros(rng, L, cfg.n_macros, cfg.macro_frac)
    w = np.concatenate([w_mov, fw]).astype(np.float32)
    h = np.concatenate([h_mov, fh]).astype(np.float32)
    net_ptr, pin_cell, dx, dy = netlist(rng, cfg.m, cfg.E, w_mov, h_mov, cfg.degree_uniform)
    _macro_pins(rng, net_ptr, pin_cell, dx, dy, cfg.m, fw, fh)
    x, y = gaussian_start(rng, region, w_mov, h_mov)
    return Instance(name=cfg.name, region=region, n=cfg.n,
                    target_density=cfg.target_density,
                    gamma=float(cfg.gamma_bins * cfg.wb),
                    m_mov=cfg.m, m_fix=int(fw.shape[0]), w=w, h=h,
                    fix_x=fx, fix_y=fy, net_ptr=net_ptr, pin_cell=pin_cell,
                    pin_dx=dx, pin_dy=dy, x=x, y=y, seed=seed)


def scaled_config(base: str, m: int, name: str | None = None) -> Config:
    """A config with the base's distributions and density, resized to m cells."""
    b = CONFIGS[base]
    s = m / b.m
    n = 1 << max(4, math.ceil(math.log2(math.sqrt(m))))
    wb = b.wb
    return Config(name or f"{base}_m{m}", wb * n, n, m, max(1, int(round(b.E * s))),
                  max(0, int(round(b.n_macros * s))) if b.n_macros else 0,
                  b.macro_frac, b.target_density, b.gamma_bins,
                  b.tiny_widths, b.degree_uniform, b.index)


def serving_job_config(rng: np.random.Generator, m_lo: int = 5_000, m_hi: int = 500_000,
                       util: float = 0.6, macro_frac: float = 0.12) -> Config:
    """One job of the serving stream: m log-uniform in [m_lo, m_hi], E = 1.05 m,
    n = 2^ceil(log2 sqrt m), w_b the smallest multiple of 0.5 with utilisation
    (movable area / free area) at most `util`, macro count proportional to m."""
    m = int(round(math.exp(rng.uniform(math.log(m_lo), math.log(m_hi)))))
    n = 1 << max(4, math.ceil(math.log2(math.sqrt(m))))
    mean_area = 2.4
    wb = 0.5
    while True:
        L = wb * n
        free = L * L * (1.0 - macro_frac)
        if m * mean_area / free <= util:
            break
        wb += 0.5
    n_mac = max(1, int(round(40 * m / 210_000)))
    return Config(f"job_m{m}", wb * n, n, m, int(round(1.05 * m)), n_mac, macro_frac,
                  0.9, 0.5, index=4)


def random_cells(rng: np.random.Generator, m: int, region, wmax: float = 6.0,
                 hmax: float = 2.0, outside: float = 0.0):
    """Free-form random cells for property tests: centres uniform in the region
    enlarged by `outside` on every side, sizes uniform in (0, wmax] x (0, hmax]."""
    x0, y0, x1, y1 = region
    x = rng.uniform(x0 - outside, x1 + outside, size=m).astype(np.float32)
    y = rng.uniform(y0 - outside, y1 + outside, size=m).astype(np.float32)
    w = rng.uniform(0.05, wmax, size=m).astype(np.float32)
    h = rng.uniform(0.05, hmax, size=m).astype(np.float32)
    return x, y, w, h


def with_fillers(inst: Instance, count: int, filler_w: float, filler_h: float,
                 seed: int | None = None) -> Instance:
    """A copy of inst with `count` pin-less movable cells of size
    filler_w x filler_h appended after the movable cells, at seeded uniform
    positions inside the region (the count and size come from the caller).
    Fixed-cell pin indices shift by count."""
    rng = np.random.default_rng(1312 + 7919 if seed is None else seed)
    x0, y0, x1, y1 = inst.region
    m = inst.m_mov
    fw = np.full(count, filler_w, np.float32)
    fh = np.full(count, filler_h, np.float32)
    fxs = rng.uniform(x0 + 0.5 * filler_w, x1 - 0.5 * filler_w, count).astype(np.float32)
    fys = rng.uniform(y0 + 0.5 * filler_h, y1 - 0.5 * filler_h, count).astype(np.float32)
    pc = inst.pin_cell.astype(np.int64)
    pc = np.where(pc >= m, pc + count, pc).astype(np.int32)
    return Instance(name=inst.name + "+fillers", region=inst.region, n=inst.n,
                    target_density=inst.target_density, gamma=inst.gamma,
                    m_mov=m + count, m_fix=inst.m_fix,
                    w=np.concatenate([inst.w[:m], fw, inst.w[m:]]),
                    h=np.concatenate([inst.h[:m], fh, inst.h[m:]]),
                    fix_x=inst.fix_x, fix_y=inst.fix_y, net_ptr=inst.net_ptr, pin_cell=pc,
                    pin_dx=inst.pin_dx, pin_dy=inst.pin_dy,
                    x=np.concatenate([inst.x, fxs]), y=np.concatenate([inst.y, fys]),
                    seed=inst.seed, extra=dict(inst.extra, fillers=count))
