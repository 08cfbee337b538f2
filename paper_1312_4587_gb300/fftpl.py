"""Python binding of libfftpl (include/fftpl.h): argument marshalling only.

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: positions and gradients are torch CUDA tensors
(float32, contiguous) whose device pointers are passed through; host arrays
for fftpl_create are numpy.  Borrowed device maps come back as zero-copy
torch views through the CUDA array interface.

The library must be built (``__graft_entry__.build()``); importing the
functions without it raises, and nothing falls back to another
implementation.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfftpl.so")

FFTPL_OK, FFTPL_EINVAL, FFTPL_ENOMEM, FFTPL_ECUDA, FFTPL_ETIMEOUT, FFTPL_ESTATE, \
    FFTPL_EUNSUPPORTED = range(7)
STATUS_NAMES = {0: "FFTPL_OK", 1: "FFTPL_EINVAL", 2: "FFTPL_ENOMEM", 3: "FFTPL_ECUDA",
                4: "FFTPL_ETIMEOUT", 5: "FFTPL_ESTATE", 6: "FFTPL_EUNSUPPORTED"}
FFTPL_SOLVE_FFT, FFTPL_SOLVE_TC_BF16X3, FFTPL_SOLVE_TC_RADIX = 0, 1, 2
FFTPL_TC_MIN_N = 128
FFTPL_TCR_MIN_N = 256
FFTPL_WL_WA, FFTPL_WL_LSE = 0, 1
FFTPL_OPT_NESTEROV, FFTPL_OPT_CG = 0, 1
FFTPL_NUM_STAGES = 8
STAGES = ["scatter", "rows_fwd", "cols", "rows_inv", "wa", "cells", "step", "reserved"]


class FFTPLError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class fftpl_region(C.Structure):
    _fields_ = [("x0", C.c_double), ("y0", C.c_double), ("x1", C.c_double), ("y1", C.c_double)]


class fftpl_cells(C.Structure):
    _fields_ = [("m_mov", C.c_int32), ("m_fix", C.c_int32), ("w", C.c_void_p),
                ("h", C.c_void_p), ("fix_x", C.c_void_p), ("fix_y", C.c_void_p)]


class fftpl_nets(C.Structure):
    _fields_ = [("E", C.c_int32), ("net_ptr", C.c_void_p)]


class fftpl_pins(C.Structure):
    _fields_ = [("P", C.c_int64), ("pin_cell", C.c_void_p), ("dx", C.c_void_p),
                ("dy", C.c_void_p)]


class fftpl_options(C.Structure):
    _fields_ = [("target_density", C.c_double), ("solve_path", C.c_int32),
                ("deterministic", C.c_int32), ("lambda0", C.c_double),
                ("gamma_fixed", C.c_double), ("dw_ref", C.c_double),
                ("alpha_max0_bins", C.c_double), ("tau_stop", C.c_double),
                ("stop_on_tau", C.c_int32), ("use_graphs", C.c_int32),
                ("wirelength", C.c_int32), ("optimizer", C.c_int32),
                ("helmholtz_eps", C.c_double), ("alpha_max_cap_bins", C.c_double)]


class fftpl_eval_report(C.Structure):
    _fields_ = [("N", C.c_double), ("W", C.c_double), ("hpwl", C.c_double), ("tau", C.c_double),
                ("gN_l1", C.c_double), ("gW_l1", C.c_double), ("charge", C.c_double),
                ("mov_area", C.c_double)]

    def as_dict(self):
        return {k: float(getattr(self, k)) for k, _ in self._fields_}


class fftpl_iter_record(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("W", "hpwl", "N", "tau", "lambda_", "gamma", "alpha",
                                          "step_max")]

    def as_dict(self):
        d = {k: float(getattr(self, k)) for k, _ in self._fields_}
        d["lam"] = d.pop("lambda_")
        return d


class fftpl_server_options(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_int32),
                ("iters_per_tick", C.c_int32), ("deterministic", C.c_int32),
                ("dry_run", C.c_int32), ("workers", C.c_int32), ("reserved", C.c_int32 * 3)]


class fftpl_job_info(C.Structure):
    _fields_ = [("id", C.c_int64), ("state", C.c_int32), ("iters_done", C.c_int32),
                ("m_mov", C.c_int32), ("n", C.c_int32), ("t_submit", C.c_double),
                ("t_admit", C.c_double), ("t_done", C.c_double), ("hpwl", C.c_double),
                ("tau", C.c_double), ("device_bytes", C.c_size_t)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class fftpl_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("failed", C.c_int64),
                ("active", C.c_int32), ("queued", C.c_int32), ("peak_active", C.c_int32),
                ("peak_device_bytes", C.c_size_t), ("wall_s", C.c_double),
                ("jobs_per_s", C.c_double), ("iter_p50_ms", C.c_double),
                ("iter_p99_ms", C.c_double), ("job_p50_ms", C.c_double),
                ("job_p99_ms", C.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


FFTPL_JOB_QUEUED, FFTPL_JOB_ACTIVE, FFTPL_JOB_DONE, FFTPL_JOB_FAILED = range(4)

_lib = None
_P = C.c_void_p
_H = C.c_void_p


def lib():
    """The loaded libfftpl.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        S = C.c_int
        sig = {
            "fftpl_version": (C.c_int32, []),
            "fftpl_default_options": (None, [_P]),
            "fftpl_create": (S, [_P, C.c_int32, _P, _P, _P, _P, _P, _P]),
            "fftpl_destroy": (None, [_H]),
            "fftpl_last_error": (C.c_char_p, [_H]),
            "fftpl_check": (S, [_H]),
            "fftpl_device_bytes": (C.c_size_t, [_H]),
            "fftpl_density": (S, [_H, _P, _P, _P, _P, _P]),
            "fftpl_density_adjoint": (S, [_H, _P, _P, _P, _P, _P]),
            "fftpl_wa": (S, [_H, _P, _P, C.c_float, _P, _P, _P]),
            "fftpl_energy": (S, [_H, _P, _P, _P]),
            "fftpl_gather": (S, [_H, _P, _P, C.c_int32, _P, _P]),
            "fftpl_eval": (S, [_H, _P, _P, C.c_float, _P, _P, _P, _P, _P]),
            "fftpl_eval_host": (S, [_H, _P, _P, C.c_float, _P, _P, _P, _P, _P]),
            "fftpl_report": (S, [_H, _P]),
            "fftpl_fields": (S, [_H, _P, _P, _P, _P]),
            "fftpl_fields_q": (S, [_H, _P]),
            "fftpl_bin_ranges": (S, [_H, _P, _P, _P, _P]),
            "fftpl_place_init": (S, [_H, _P, _P]),
            "fftpl_step": (S, [_H, C.c_int32, _P, _P]),
            "fftpl_place_positions": (S, [_H, _P, _P]),
            "fftpl_state_save": (S, [_H, _P, _P]),
            "fftpl_state_load": (S, [_H, _P, C.c_size_t]),
            "fftpl_set_profiling": (S, [_H, C.c_int32]),
            "fftpl_stage_times": (S, [_H, _P, _P, C.c_int32]),
            "fftpl_launch_count": (C.c_int64, [_H]),
            "fftpl_debug_fail_alloc_after": (None, [C.c_int32]),
            "fftpl_debug_transpose_stores": (S, [_H, C.c_int32]),
            "fftpl_fillers": (S, [_P, _P, C.c_double, _P, _P, _P]),
            "fftpl_debug_tc_gemm": (S, [_P, _P, _P, _P, C.c_int32, C.c_int32, C.c_int32, _P,
                                        C.c_int32, C.c_int32, _P, _P]),
            "fftpl_solve_noalloc": (S, [_P, C.c_int32, C.c_double, C.c_double, _P, _P, _P, _P, _P]),
            "fftpl_server_default_options": (None, [_P]),
            "fftpl_estimate_bytes": (C.c_size_t, [C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                                  C.c_int64, C.c_int32, C.c_int32]),
            "fftpl_server_create": (S, [_P, _P]),
            "fftpl_server_destroy": (None, [_P]),
            "fftpl_server_submit": (S, [_P, _P, C.c_int32, _P, _P, _P, _P, _P, _P, C.c_int32, _P]),
            "fftpl_server_tick": (S, [_P, _P, _P]),
            "fftpl_server_job": (S, [_P, C.c_int64, _P, _P, _P]),
            "fftpl_server_report": (S, [_P, _P]),
            "fftpl_server_set_clock": (S, [_P, C.c_double]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(status, h=None):
    if status != FFTPL_OK:
        msg = lib().fftpl_last_error(h)
        raise FFTPLError(status, msg.decode() if msg else "")


def _dptr(t):
    """Device pointer of a float32/int32 contiguous CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("expected a contiguous CUDA tensor")
    return C.c_void_p(t.data_ptr())


def _hptr(a, dtype):
    return C.c_void_p(a.ctypes.data) if a is not None and a.size else None


class _DeviceView:
    """Exposes a borrowed device pointer through the CUDA array interface."""

    def __init__(self, ptr, shape, typestr):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr,
                                         "data": (int(ptr), False), "version": 3,
                                         "strides": None}


def _view(ptr, shape, typestr="<f4"):
    import torch
    return torch.as_tensor(_DeviceView(ptr, shape, typestr), device="cuda")


# ---------------------------------------------------------------- entry points

def fftpl_version():
    return int(lib().fftpl_version())


def fftpl_default_options(**overrides):
    o = fftpl_options()
    lib().fftpl_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def fftpl_create(region, n, w, h, m_mov, fix_x, fix_y, net_ptr, pin_cell, pin_dx, pin_dy,
                 options=None, stream=None):
    """Creates a handle; host numpy arrays are deep-copied to the device."""
    w = np.ascontiguousarray(w, np.float32)
    h = np.ascontiguousarray(h, np.float32)
    m_fix = int(w.shape[0] - m_mov)
    fix_x = np.ascontiguousarray(fix_x if fix_x is not None else np.zeros(0), np.float32)
    fix_y = np.ascontiguousarray(fix_y if fix_y is not None else np.zeros(0), np.float32)
    net_ptr = np.ascontiguousarray(net_ptr, np.int32)
    pin_cell = np.ascontiguousarray(pin_cell, np.int32)
    pin_dx = np.ascontiguousarray(pin_dx, np.float32)
    pin_dy = np.ascontiguousarray(pin_dy, np.float32)
    R = fftpl_region(*[float(v) for v in region])
    cells = fftpl_cells(int(m_mov), m_fix, _hptr(w, 0), _hptr(h, 0), _hptr(fix_x, 0),
                        _hptr(fix_y, 0))
    nets = fftpl_nets(int(net_ptr.shape[0] - 1), C.c_void_p(net_ptr.ctypes.data))
    pins = fftpl_pins(int(pin_cell.shape[0]), _hptr(pin_cell, 0), _hptr(pin_dx, 0),
                      _hptr(pin_dy, 0))
    if options is None:
        options = fftpl_default_options()
    if stream is None:
        try:
            import torch
            stream = torch.cuda.current_stream().cuda_stream if torch.cuda.is_available() else 0
        except Exception:
            stream = 0
    out = C.c_void_p()
    st = lib().fftpl_create(C.byref(R), C.c_int32(int(n)), C.byref(cells), C.byref(nets),
                            C.byref(pins), C.byref(options), C.c_void_p(int(stream or 0)),
                            C.byref(out))
    _check(st, None)
    return out


def fftpl_destroy(h):
    if h:
        lib().fftpl_destroy(h)


def fftpl_last_error(h=None):
    s = lib().fftpl_last_error(h)
    return s.decode() if s else ""


def fftpl_check(h):
    _check(lib().fftpl_check(h), h)


def fftpl_device_bytes(h):
    return int(lib().fftpl_device_bytes(h))


def fftpl_density(h, x, y, gx=None, gy=None, sync=True):
    N = C.c_double(0.0)
    _check(lib().fftpl_density(h, _dptr(x), _dptr(y), C.byref(N) if sync else None,
                               _dptr(gx), _dptr(gy)), h)
    return float(N.value) if sync else None


def fftpl_density_adjoint(h, x, y, gx=None, gy=None, sync=True):
    N = C.c_double(0.0)
    _check(lib().fftpl_density_adjoint(h, _dptr(x), _dptr(y), C.byref(N) if sync else None,
                                       _dptr(gx), _dptr(gy)), h)
    return float(N.value) if sync else None


def fftpl_energy(h, x, y, sync=True):
    N = C.c_double(0.0)
    _check(lib().fftpl_energy(h, _dptr(x), _dptr(y), C.byref(N) if sync else None), h)
    return float(N.value) if sync else None


def fftpl_gather(h, x, y, gx, gy, mode=0):
    _check(lib().fftpl_gather(h, _dptr(x), _dptr(y), C.c_int32(int(mode)), _dptr(gx), _dptr(gy)),
           h)


def fftpl_wa(h, x, y, gamma, gx=None, gy=None, sync=True):
    W = C.c_double(0.0)
    _check(lib().fftpl_wa(h, _dptr(x), _dptr(y), C.c_float(gamma), C.byref(W) if sync else None,
                          _dptr(gx), _dptr(gy)), h)
    return float(W.value) if sync else None


def fftpl_eval(h, x, y, gamma, gNx=None, gNy=None, gWx=None, gWy=None, sync=True):
    rep = fftpl_eval_report()
    _check(lib().fftpl_eval(h, _dptr(x), _dptr(y), C.c_float(gamma), _dptr(gNx), _dptr(gNy),
                            _dptr(gWx), _dptr(gWy), C.byref(rep) if sync else None), h)
    return rep.as_dict() if sync else None


def fftpl_eval_host(h, x, y, gamma, gNx=None, gNy=None, gWx=None, gWy=None):
    """Host (CPU tensors or numpy, float32 contiguous; pinned is fastest)."""
    def hp(a):
        if a is None:
            return None
        if hasattr(a, "data_ptr"):
            return C.c_void_p(a.data_ptr())
        return C.c_void_p(a.ctypes.data)
    rep = fftpl_eval_report()
    _check(lib().fftpl_eval_host(h, hp(x), hp(y), C.c_float(gamma), hp(gNx), hp(gNy), hp(gWx),
                                 hp(gWy), C.byref(rep)), h)
    return rep.as_dict()


def fftpl_report(h):
    rep = fftpl_eval_report()
    _check(lib().fftpl_report(h, C.byref(rep)), h)
    return rep.as_dict()


def fftpl_fields(h, n):
    """Borrowed views {rho, psi, ex, ey} ([n, n] float32 CUDA tensors)."""
    ptrs = [C.c_void_p() for _ in range(4)]
    _check(lib().fftpl_fields(h, *[C.byref(p) for p in ptrs]), h)
    return {k: _view(p.value, (n, n)) for k, p in zip(("rho", "psi", "ex", "ey"), ptrs)}


def fftpl_fields_q(h, n):
    p = C.c_void_p()
    _check(lib().fftpl_fields_q(h, C.byref(p)), h)
    return _view(p.value, (n, n), "<i8")


def fftpl_bin_ranges(h, x, y, ranges):
    pairs = C.c_int64(0)
    _check(lib().fftpl_bin_ranges(h, _dptr(x), _dptr(y), _dptr(ranges), C.byref(pairs)), h)
    return int(pairs.value)


def fftpl_place_init(h, x0, y0):
    _check(lib().fftpl_place_init(h, _dptr(x0), _dptr(y0)), h)


def fftpl_step(h, iters, records=True):
    recs = (fftpl_iter_record * max(int(iters), 1))() if records else None
    ran = C.c_int32(0)
    _check(lib().fftpl_step(h, C.c_int32(int(iters)), recs, C.byref(ran)), h)
    rows = [recs[k].as_dict() for k in range(ran.value)] if records else []
    return rows, int(ran.value)


def fftpl_place_positions(h, x, y):
    _check(lib().fftpl_place_positions(h, _dptr(x), _dptr(y)), h)


def fftpl_state_save(h):
    n = C.c_size_t(0)
    _check(lib().fftpl_state_save(h, None, C.byref(n)), h)
    buf = C.create_string_buffer(n.value)
    _check(lib().fftpl_state_save(h, buf, C.byref(n)), h)
    return buf.raw[: n.value]


def fftpl_state_load(h, data: bytes):
    buf = C.create_string_buffer(data, len(data))
    _check(lib().fftpl_state_load(h, buf, C.c_size_t(len(data))), h)


def fftpl_set_profiling(h, on):
    _check(lib().fftpl_set_profiling(h, C.c_int32(1 if on else 0)), h)


def fftpl_stage_times(h, reset=False):
    ms = (C.c_double * FFTPL_NUM_STAGES)()
    ln = (C.c_int64 * FFTPL_NUM_STAGES)()
    _check(lib().fftpl_stage_times(h, ms, ln, C.c_int32(1 if reset else 0)), h)
    return list(ms), list(ln)


def fftpl_launch_count(h):
    return int(lib().fftpl_launch_count(h))


def fftpl_solve_noalloc(rho, n, Lx, Ly, psi, ex, ey, want_N=False, stream=None):
    """Allocation-free solve of a device density map rho ([n, n] float32 CUDA
    tensor) into caller-owned psi, ex, ey; returns N if want_N."""
    import torch
    for name, t in (("rho", rho), ("psi", psi), ("ex", ex), ("ey", ey)):
        if t.dtype != torch.float32 or t.numel() < int(n) * int(n):
            raise ValueError(f"fftpl_solve_noalloc: {name} must be float32 with at least "
                             f"n*n = {int(n) * int(n)} elements")
    N = C.c_double(0.0)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().fftpl_solve_noalloc(_dptr(rho), C.c_int32(int(n)), C.c_double(Lx),
                                     C.c_double(Ly), _dptr(psi), _dptr(ex), _dptr(ey),
                                     C.byref(N) if want_N else None, C.c_void_p(int(stream or 0))),
           None)
    return float(N.value) if want_N else None


def fftpl_server_default_options(**overrides):
    o = fftpl_server_options()
    lib().fftpl_server_default_options(C.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


def fftpl_estimate_bytes(n, m_mov, m_fix, E, P, iters, deterministic=0):
    return int(lib().fftpl_estimate_bytes(int(n), int(m_mov), int(m_fix), int(E), int(P),
                                          int(iters), int(deterministic)))


def fftpl_server_create(options=None):
    out = C.c_void_p()
    o = options if options is not None else fftpl_server_default_options()
    _check(lib().fftpl_server_create(C.byref(o), C.byref(out)), None)
    return out


def fftpl_server_destroy(s):
    if s:
        lib().fftpl_server_destroy(s)


def fftpl_server_submit(s, region, n, w, h, m_mov, fix_x, fix_y, net_ptr, pin_cell, pin_dx,
                        pin_dy, x0, y0, iters, options=None):
    """Queues a job (host numpy arrays, deep-copied); returns its id."""
    w = np.ascontiguousarray(w, np.float32); h = np.ascontiguousarray(h, np.float32)
    m_fix = int(w.shape[0] - m_mov)
    fix_x = np.ascontiguousarray(fix_x if fix_x is not None else np.zeros(0), np.float32)
    fix_y = np.ascontiguousarray(fix_y if fix_y is not None else np.zeros(0), np.float32)
    net_ptr = np.ascontiguousarray(net_ptr, np.int32)
    pin_cell = np.ascontiguousarray(pin_cell, np.int32)
    pin_dx = np.ascontiguousarray(pin_dx, np.float32); pin_dy = np.ascontiguousarray(pin_dy, np.float32)
    x0 = np.ascontiguousarray(x0, np.float32); y0 = np.ascontiguousarray(y0, np.float32)
    R = fftpl_region(*[float(v) for v in region])
    cells = fftpl_cells(int(m_mov), m_fix, _hptr(w, 0), _hptr(h, 0), _hptr(fix_x, 0), _hptr(fix_y, 0))
    nets = fftpl_nets(int(net_ptr.shape[0] - 1), C.c_void_p(net_ptr.ctypes.data))
    pins = fftpl_pins(int(pin_cell.shape[0]), _hptr(pin_cell, 0), _hptr(pin_dx, 0), _hptr(pin_dy, 0))
    o = options if options is not None else fftpl_default_options()
    jid = C.c_int64(0)
    _check(lib().fftpl_server_submit(s, C.byref(R), C.c_int32(int(n)), C.byref(cells),
                                     C.byref(nets), C.byref(pins), C.byref(o), _hptr(x0, 0),
                                     _hptr(y0, 0), C.c_int32(int(iters)), C.byref(jid)), None)
    return int(jid.value)


def fftpl_server_tick(s):
    a = C.c_int32(0); q = C.c_int32(0)
    _check(lib().fftpl_server_tick(s, C.byref(a), C.byref(q)), None)
    return int(a.value), int(q.value)


def fftpl_server_job(s, jid, m_mov=None):
    """(info dict, x, y); x and y are numpy arrays once the job is done."""
    info = fftpl_job_info()
    _check(lib().fftpl_server_job(s, C.c_int64(int(jid)), C.byref(info), None, None), None)
    x = y = None
    if info.state == FFTPL_JOB_DONE and m_mov:
        x = np.empty(m_mov, np.float32); y = np.empty(m_mov, np.float32)
        _check(lib().fftpl_server_job(s, C.c_int64(int(jid)), None, _hptr(x, 0), _hptr(y, 0)), None)
    return info.as_dict(), x, y


def fftpl_server_report(s):
    st = fftpl_server_stats()
    _check(lib().fftpl_server_report(s, C.byref(st)), None)
    return st.as_dict()


def fftpl_server_set_clock(s, now_s):
    _check(lib().fftpl_server_set_clock(s, C.c_double(float(now_s))), None)


def fftpl_fillers(region, w, h, m_mov, fix_x=None, fix_y=None, target_density=1.0):
    """Filler count and size for an instance (host arrays): (count, w, h)."""
    w = np.ascontiguousarray(w, np.float32)
    h = np.ascontiguousarray(h, np.float32)
    m_fix = int(w.shape[0]) - int(m_mov)
    fx = np.ascontiguousarray(fix_x if fix_x is not None else np.zeros(0), np.float32)
    fy = np.ascontiguousarray(fix_y if fix_y is not None else np.zeros(0), np.float32)
    R = fftpl_region(*[float(v) for v in region])
    cells = fftpl_cells(int(m_mov), m_fix, _hptr(w, 0), _hptr(h, 0), _hptr(fx, 0), _hptr(fy, 0))
    cnt = C.c_int64(0); a = C.c_float(0.0); b = C.c_float(0.0)
    _check(lib().fftpl_fillers(C.byref(R), C.byref(cells), C.c_double(target_density),
                               C.byref(cnt), C.byref(a), C.byref(b)), None)
    return int(cnt.value), float(a.value), float(b.value)


def fftpl_debug_fail_alloc_after(k):
    lib().fftpl_debug_fail_alloc_after(C.c_int32(int(k)))


def fftpl_debug_transpose_stores(h, tma):
    _check(lib().fftpl_debug_transpose_stores(h, C.c_int32(1 if tma else 0)), h)


def fftpl_debug_tc_gemm(a_hi, a_lo, b_hi, b_lo, d, err, nsplit=3, no_loads=0, stream=None):
    """d[M][N] = (a_hi + a_lo) @ (b_hi + b_lo)^T on the tensor cores: bf16 CUDA
    tensors a_* [M][K], b_* [N][K], float32 d [M][N], int32 err [1]."""
    M, K = a_hi.shape
    N = b_hi.shape[0]
    if stream is None:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    _check(lib().fftpl_debug_tc_gemm(_dptr(a_hi), _dptr(a_lo), _dptr(b_hi), _dptr(b_lo),
                                     C.c_int32(M), C.c_int32(N), C.c_int32(K), _dptr(d),
                                     C.c_int32(nsplit), C.c_int32(no_loads), _dptr(err),
                                     C.c_void_p(int(stream or 0))), None)


# ---------------------------------------------------------------- convenience

class Problem:
    """Owns one handle for a placement instance (an object with the fields of
    a seeded instance: region, n, w, h, m_mov, fix_x, fix_y, net_ptr,
    pin_cell, pin_dx, pin_dy, target_density)."""

    def __init__(self, inst, stream=None, **opts):
        o = fftpl_default_options(target_density=float(getattr(inst, "target_density", 1.0)))
        for k, v in opts.items():
            setattr(o, k, v)
        self.inst = inst
        self.n = int(inst.n)
        self.m = int(inst.m_mov)
        self.options = o
        self.h = fftpl_create(inst.region, inst.n, inst.w, inst.h, inst.m_mov, inst.fix_x,
                              inst.fix_y, inst.net_ptr, inst.pin_cell, inst.pin_dx, inst.pin_dy,
                              o, stream)

    def close(self):
        if self.h:
            fftpl_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
