"""FP64 CPU oracle for the FFTPL objective-gradient evaluation (test infrastructure).

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The library path never does: it shares
no code with the CUDA kernels and fails loudly without them.

The arithmetic lives in ``fftpl_oracle.c`` (plain loops in FP64, one function
per step of the method, each citing the paper's equation).  This module
compiles it with gcc and wraps it with ctypes so that tests can pass numpy
arrays.  Pins of every function against closed forms, invariants and brute
force are in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fftpl_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into oracle/liboracle.so (gcc, OpenMP when available)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.run(base[:4] + ["-fopenmp"] + base[4:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB)
    return _LIB


class Region(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double)]


class EvalOut(C.Structure):
    _fields_ = [("N", C.c_double), ("W", C.c_double), ("hpwl", C.c_double),
                ("tau", C.c_double), ("total_mov_area", C.c_double),
                ("gN_l1", C.c_double), ("gW_l1", C.c_double)]


class IterRec(C.Structure):
    _fields_ = [("W", C.c_double), ("hpwl", C.c_double), ("N", C.c_double),
                ("tau", C.c_double), ("lambda_", C.c_double), ("gamma", C.c_double),
                ("alpha", C.c_double), ("step_max", C.c_double)]


class PointOut(C.Structure):
    _fields_ = [("W", C.c_double), ("hpwl", C.c_double), ("N", C.c_double),
                ("tau", C.c_double), ("gN_l1", C.c_double), ("gW_l1", C.c_double)]


# void f(void* ctx, const double* v, double gamma, double* gW, double* gN, PointOut* out)
ObjectiveFn = C.CFUNCTYPE(None, C.c_void_p, C.POINTER(C.c_double), C.c_double,
                          C.POINTER(C.c_double), C.POINTER(C.c_double), C.POINTER(PointOut))


class LoopOpts(C.Structure):
    _fields_ = [("lambda0", C.c_double), ("gamma_fixed", C.c_double),
                ("dw_ref", C.c_double), ("alpha_max0_bins", C.c_double),
                ("stop_on_tau", C.c_int), ("tau_stop", C.c_double),
                ("wirelength", C.c_int), ("helmholtz_eps", C.c_double),
                ("alpha_max_cap_bins", C.c_double)]

# wirelength models
WL_WA, WL_LSE = 0, 1


_P = C.c_void_p


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB)
            L.orc_bin_ranges.restype = C.c_int64
            L.orc_energy.restype = C.c_double
            L.orc_overflow.restype = C.c_double
            L.orc_wa.restype = C.c_double
            L.orc_wl.restype = C.c_double
            L.orc_mu.restype = C.c_double
            L.orc_mu.argtypes = [C.c_double, C.c_double]
            L.orc_gamma.restype = C.c_double
            L.orc_gamma.argtypes = [C.c_double, C.c_double]
            L.orc_nesterov_a.restype = C.c_double
            L.orc_nesterov_a.argtypes = [C.c_double]
            L.orc_nesterov.restype = C.c_int
            L.orc_nesterov_run.restype = C.c_int
            L.orc_nesterov_run.argtypes = [C.c_int, _P, _P, _P, C.c_double, ObjectiveFn,
                                           C.c_void_p, C.POINTER(LoopOpts), C.c_int, _P]
            L.orc_cg.restype = C.c_int
            L.orc_num_threads.restype = C.c_int
            _lib = L
    return _lib


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _ptr(a):
    return a.ctypes.data_as(_P) if a is not None else None


def _region(region):
    return Region(*[float(v) for v in region])


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(t: int) -> None:
    lib().orc_set_num_threads(C.c_int(int(t)))


# ----------------------------------------------------------------------------
# wrappers
# ----------------------------------------------------------------------------

def bin_ranges(region, n, x, y, w, h):
    """(ranges int32 [m,4] = ilo, ihi, jlo, jhi; pair count)."""
    x, y, w, h = map(_f32, (x, y, w, h))
    m = x.shape[0]
    out = np.zeros((m, 4), dtype=np.int32)
    R = _region(region)
    pairs = lib().orc_bin_ranges(C.byref(R), C.c_int(n), C.c_int(m), _ptr(x), _ptr(y),
                                 _ptr(w), _ptr(h), _ptr(out))
    return out, int(pairs)


def overlap_map(region, n, x, y, w, h):
    x, y, w, h = map(_f32, (x, y, w, h))
    out = np.zeros((n, n), dtype=np.float64)
    R = _region(region)
    lib().orc_overlap_map(C.byref(R), C.c_int(n), C.c_int(x.shape[0]), _ptr(x), _ptr(y),
                          _ptr(w), _ptr(h), _ptr(out))
    return out


def overlap_map_q(region, n, x, y, w, h):
    x, y, w, h = map(_f32, (x, y, w, h))
    out = np.zeros((n, n), dtype=np.int64)
    R = _region(region)
    lib().orc_overlap_map_q(C.byref(R), C.c_int(n), C.c_int(x.shape[0]), _ptr(x), _ptr(y),
                            _ptr(w), _ptr(h), _ptr(out))
    return out


def density(region, n, rho_t, x, y, w, h, fx=None, fy=None, fw=None, fh=None):
    """(rho, movable area D, fixed area F), each [n, n] float64."""
    x, y, w, h = map(_f32, (x, y, w, h))
    m_fix = 0 if fx is None else int(np.asarray(fx).shape[0])
    fx, fy, fw, fh = (map(_f32, (fx, fy, fw, fh)) if m_fix else (None,) * 4)
    rho = np.zeros((n, n)); D = np.zeros((n, n)); F = np.zeros((n, n))
    R = _region(region)
    lib().orc_density(C.byref(R), C.c_int(n), C.c_double(rho_t), C.c_int(x.shape[0]),
                      _ptr(x), _ptr(y), _ptr(w), _ptr(h), C.c_int(m_fix),
                      _ptr(fx), _ptr(fy), _ptr(fw), _ptr(fh), _ptr(rho), _ptr(D), _ptr(F))
    return rho, D, F


def dct_coeffs(rho, keep_dc=False):
    """Eq. 10 coefficients a[v][u]; the (0,0) one zeroed unless keep_dc."""
    rho = _f64(rho)
    n = rho.shape[0]
    a = np.zeros((n, n))
    if keep_dc:
        lib().orc_dct_coeffs_dc(C.c_int(n), _ptr(rho), _ptr(a))
    else:
        lib().orc_dct_coeffs(C.c_int(n), _ptr(rho), _ptr(a))
    return a


def potential_field(a, Lx, Ly, eps=0.0):
    """psi, E_x, E_y (Eqs. 11-12); eps > 0: Helmholtz divisor w^2 + eps
    with the (0,0) mode a_00/eps (Eq. 4)."""
    a = _f64(a)
    n = a.shape[0]
    psi = np.zeros((n, n)); ex = np.zeros((n, n)); ey = np.zeros((n, n))
    lib().orc_potential_field_eps(C.c_int(n), C.c_double(Lx), C.c_double(Ly), _ptr(a),
                                  C.c_double(eps), _ptr(psi), _ptr(ex), _ptr(ey))
    return psi, ex, ey


def potential_at(a, Lx, Ly, xs, ys):
    """psi, E_x, E_y (Eqs. 11-12) at bins (ys[k], xs[k]) from coefficients a."""
    a = _f64(a)
    n = a.shape[0]
    xs = _i32(xs); ys = _i32(ys)
    k = xs.shape[0]
    psi = np.zeros(k); ex = np.zeros(k); ey = np.zeros(k)
    lib().orc_potential_at(C.c_int(n), C.c_double(Lx), C.c_double(Ly), _ptr(a), C.c_int(k),
                           _ptr(xs), _ptr(ys), _ptr(psi), _ptr(ex), _ptr(ey))
    return psi, ex, ey


def solve(rho, Lx, Ly, eps=0.0):
    """rho -> (a, psi, E_x, E_y) by the explicit cosine sums of Eqs. 9-12
    (eps > 0: the Helmholtz equation of Eq. 4)."""
    a = dct_coeffs(rho, keep_dc=eps > 0)
    psi, ex, ey = potential_field(a, Lx, Ly, eps)
    return a, psi, ex, ey


def energy(rho, psi, Ab):
    rho, psi = _f64(rho), _f64(psi)
    return float(lib().orc_energy(C.c_int(rho.shape[0]), C.c_double(Ab), _ptr(rho), _ptr(psi)))


def gather(region, n, x, y, w, h, ex, ey):
    x, y, w, h = map(_f32, (x, y, w, h))
    ex, ey = _f64(ex), _f64(ey)
    m = x.shape[0]
    gx = np.zeros(m); gy = np.zeros(m)
    R = _region(region)
    lib().orc_gather(C.byref(R), C.c_int(n), C.c_int(m), _ptr(x), _ptr(y), _ptr(w), _ptr(h),
                     _ptr(ex), _ptr(ey), _ptr(gx), _ptr(gy))
    return gx, gy


def adjoint(region, n, x, y, w, h, psi):
    x, y, w, h = map(_f32, (x, y, w, h))
    psi = _f64(psi)
    m = x.shape[0]
    gx = np.zeros(m); gy = np.zeros(m)
    R = _region(region)
    lib().orc_adjoint(C.byref(R), C.c_int(n), C.c_int(m), _ptr(x), _ptr(y), _ptr(w), _ptr(h),
                      _ptr(psi), _ptr(gx), _ptr(gy))
    return gx, gy


def overflow(D, F, Ab, rho_t, total_mov_area):
    D = _f64(D)
    F = None if F is None else _f64(F)
    return float(lib().orc_overflow(C.c_int(D.shape[0]), C.c_double(Ab), C.c_double(rho_t),
                                    _ptr(D), _ptr(F), C.c_double(total_mov_area)))


def wa(net_ptr, pin_cell, dx, dy, m_mov, x, y, gamma, fx=None, fy=None, per_pin=False,
       model=WL_WA):
    """Smoothed wirelength: weighted average (Eq. 3, model WL_WA) or
    log-sum-exp (WL_LSE).  Returns dict with W (sum), hpwl, net_w [E],
    gcx/gcy [m_mov] and, if per_pin, gpx/gpy [P]."""
    net_ptr, pin_cell = _i32(net_ptr), _i32(pin_cell)
    dx, dy, x, y = map(_f32, (dx, dy, x, y))
    fx = _f32(fx) if fx is not None else np.zeros(1, np.float32)
    fy = _f32(fy) if fy is not None else np.zeros(1, np.float32)
    E = net_ptr.shape[0] - 1
    P = pin_cell.shape[0]
    net_w = np.zeros(max(E, 1))
    gcx = np.zeros(max(m_mov, 1)); gcy = np.zeros(max(m_mov, 1))
    gpx = np.zeros(max(P, 1)) if per_pin else None
    gpy = np.zeros(max(P, 1)) if per_pin else None
    hp = C.c_double(0.0)
    W = lib().orc_wl(C.c_int(model), C.c_int(E), _ptr(net_ptr), _ptr(pin_cell), _ptr(dx), _ptr(dy),
                     C.c_int(m_mov), _ptr(x), _ptr(y), _ptr(fx), _ptr(fy), C.c_double(gamma),
                     _ptr(net_w), _ptr(gpx), _ptr(gpy), _ptr(gcx), _ptr(gcy), C.byref(hp))
    out = dict(W=float(W), hpwl=float(hp.value), net_w=net_w[:E], gcx=gcx[:m_mov],
               gcy=gcy[:m_mov])
    if per_pin:
        out["gpx"], out["gpy"] = gpx[:P], gpy[:P]
    return out


def mu(dW, dW_ref):
    return float(lib().orc_mu(dW, dW_ref))


def gamma_schedule(tau, wb):
    return float(lib().orc_gamma(tau, wb))


def nesterov_a(a):
    return float(lib().orc_nesterov_a(a))


def _inst_arrays(inst):
    m, k = inst.m_mov, inst.m_fix
    w, h = _f32(inst.w), _f32(inst.h)
    fw = w[m:] if k else None
    fh = h[m:] if k else None
    return m, k, w, h, fw, fh


def eval_instance(inst, x=None, y=None, gamma=None, maps=False, wirelength=WL_WA,
                  helmholtz_eps=0.0):
    """One full objective-gradient evaluation of a synth.Instance
    (wirelength WL_WA or WL_LSE; helmholtz_eps > 0: Eq. 4 in place of Eq. 8)."""
    m, k, w, h, fw, fh = _inst_arrays(inst)
    x = _f32(inst.x if x is None else x)
    y = _f32(inst.y if y is None else y)
    gamma = inst.gamma if gamma is None else gamma
    n = inst.n
    fx = _f32(inst.fix_x) if k else None
    fy = _f32(inst.fix_y) if k else None
    net_ptr, pin_cell = _i32(inst.net_ptr), _i32(inst.pin_cell)
    dx, dy = _f32(inst.pin_dx), _f32(inst.pin_dy)
    gNx = np.zeros(m); gNy = np.zeros(m); gWx = np.zeros(m); gWy = np.zeros(m)
    mp = [np.zeros((n, n)) for _ in range(4)] if maps else [None] * 4
    out = EvalOut()
    R = _region(inst.region)
    lib().orc_eval2(C.byref(R), C.c_int(n), C.c_double(inst.target_density), C.c_int(m),
                    _ptr(x), _ptr(y), _ptr(w), _ptr(h), C.c_int(k), _ptr(fx), _ptr(fy),
                    _ptr(fw), _ptr(fh), C.c_int(net_ptr.shape[0] - 1), _ptr(net_ptr),
                    _ptr(pin_cell), _ptr(dx), _ptr(dy), C.c_double(gamma),
                    C.c_int(wirelength), C.c_double(helmholtz_eps),
                    _ptr(gNx), _ptr(gNy), _ptr(gWx), _ptr(gWy),
                   _ptr(mp[0]), _ptr(mp[1]), _ptr(mp[2]), _ptr(mp[3]), C.byref(out))
    res = dict(N=out.N, W=out.W, hpwl=out.hpwl, tau=out.tau, total_mov_area=out.total_mov_area,
               gN_l1=out.gN_l1, gW_l1=out.gW_l1, gNx=gNx, gNy=gNy, gWx=gWx, gWy=gWy)
    if maps:
        res.update(rho=mp[0], psi=mp[1], ex=mp[2], ey=mp[3])
    return res


def nesterov(inst, iters, **kw):
    """Global placement loop (Algorithm 1 with a Nesterov step).  Returns
    (x, y, records[k] dicts, iterations run)."""
    return _loop("orc_nesterov", inst, iters, **kw)


def nesterov_run(x0, lo, hi, wb, objective, iters, lambda0=0.0, gamma_fixed=1.0, dw_ref=3.5e5,
                 alpha_max0_bins=0.044, stop_on_tau=False, tau_stop=0.1, alpha_max_cap_bins=0.0):
    """The loop of orc_nesterov (Nesterov step, Section IV-A control) on an
    objective given as a Python callable objective(v, gamma) -> dict with
    gW, gN (arrays like v) and W, hpwl, N, tau, gN_l1, gW_l1 (gamma == 0 and
    no gradients asked: only tau is read).  Returns (u, records, ran)."""
    x = _f64(x0).copy()
    lo, hi = _f64(lo), _f64(hi)
    nv = x.shape[0]

    def cb(ctx, v, gamma, gW, gN, out):
        vv = np.ctypeslib.as_array(v, shape=(nv,)).copy()
        r = objective(vv, float(gamma))
        if gW:
            np.ctypeslib.as_array(gW, shape=(nv,))[:] = r["gW"]
            np.ctypeslib.as_array(gN, shape=(nv,))[:] = r["gN"]
        o = out.contents
        for k in ("W", "hpwl", "N", "tau", "gN_l1", "gW_l1"):
            setattr(o, k, float(r.get(k, 0.0)))

    fn = ObjectiveFn(cb)
    opts = LoopOpts(float(lambda0), float(gamma_fixed), float(dw_ref), float(alpha_max0_bins),
                    int(stop_on_tau), float(tau_stop), 0, 0.0, float(alpha_max_cap_bins))
    recs = (IterRec * max(iters, 1))()
    ran = lib().orc_nesterov_run(C.c_int(nv), _ptr(x), _ptr(lo), _ptr(hi), C.c_double(wb), fn,
                                 None, C.byref(opts), C.c_int(iters), C.cast(recs, _P))
    rows = [dict(W=r.W, hpwl=r.hpwl, N=r.N, tau=r.tau, lam=r.lambda_, gamma=r.gamma,
                 alpha=r.alpha, step_max=r.step_max) for r in recs[:ran]]
    return x, rows, int(ran)


def cg(inst, iters, **kw):
    """Global placement loop with the nonlinear CG step of Algorithm 1
    (Polak-Ribiere+ direction, one quadratic-fit line search in
    [0.01 a_max, a_max]).  Same arguments and results as nesterov."""
    return _loop("orc_cg", inst, iters, **kw)


def _loop(fn, inst, iters, lambda0=0.0, gamma_fixed=None, dw_ref=3.5e5, alpha_max0_bins=0.044,
          stop_on_tau=False, tau_stop=0.1, x=None, y=None, wirelength=WL_WA,
          helmholtz_eps=0.0, alpha_max_cap_bins=16.0):
    m, k, w, h, fw, fh = _inst_arrays(inst)
    x = _f32(inst.x if x is None else x).copy()
    y = _f32(inst.y if y is None else y).copy()
    fx = _f32(inst.fix_x) if k else None
    fy = _f32(inst.fix_y) if k else None
    net_ptr, pin_cell = _i32(inst.net_ptr), _i32(inst.pin_cell)
    dx, dy = _f32(inst.pin_dx), _f32(inst.pin_dy)
    gf = inst.gamma if gamma_fixed is None else gamma_fixed
    opts = LoopOpts(float(lambda0), float(gf), float(dw_ref), float(alpha_max0_bins),
                    int(stop_on_tau), float(tau_stop), int(wirelength), float(helmholtz_eps),
                    float(alpha_max_cap_bins))
    recs = (IterRec * max(iters, 1))()
    R = _region(inst.region)
    ran = getattr(lib(), fn)(C.byref(R), C.c_int(inst.n), C.c_double(inst.target_density),
                             C.c_int(m), _ptr(x), _ptr(y), _ptr(w), _ptr(h), C.c_int(k),
                             _ptr(fx), _ptr(fy), _ptr(fw), _ptr(fh),
                             C.c_int(net_ptr.shape[0] - 1), _ptr(net_ptr), _ptr(pin_cell),
                             _ptr(dx), _ptr(dy), C.byref(opts), C.c_int(iters), recs)
    rows = [dict(W=r.W, hpwl=r.hpwl, N=r.N, tau=r.tau, lam=r.lambda_, gamma=r.gamma,
                 alpha=r.alpha, step_max=r.step_max) for r in recs[:ran]]
    return x, y, rows, int(ran)


def fillers(region, w, h, m_mov, fix_x=None, fix_y=None, target_density=1.0):
    """Filler rule (Section III-B reading): (count, filler width, height)."""
    w, h = _f32(w), _f32(h)
    k = w.shape[0] - m_mov
    fx = _f32(fix_x) if k else None
    fy = _f32(fix_y) if k else None
    fw = w[m_mov:] if k else None
    fh = h[m_mov:] if k else None
    cnt = C.c_int64(0); a = C.c_float(0.0); b = C.c_float(0.0)
    R = _region(region)
    lib().orc_fillers(C.byref(R), C.c_int(m_mov), _ptr(w), _ptr(h), C.c_int(k), _ptr(fx), _ptr(fy),
                      _ptr(fw), _ptr(fh), C.c_double(target_density), C.byref(cnt), C.byref(a),
                      C.byref(b))
    return int(cnt.value), float(a.value), float(b.value)
