"""The C-ABI library builds, loads and exports every entry point that
include/fftpl.h declares; host-side validation rejects bad instances before
any device work (so these run without a GPU)."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def F():
    from paper_1312_4587_gb300 import _build
    _build.build()
    from paper_1312_4587_gb300 import fftpl
    fftpl.lib()
    return fftpl


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fftpl.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fftpl_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("fftpl_create", "fftpl_density", "fftpl_wa", "fftpl_step", "fftpl_eval",
                     "fftpl_destroy", "fftpl_fields", "fftpl_state_save", "fftpl_state_load"):
        assert required in names


def test_every_declared_symbol_is_exported(F):
    lib = ctypes.CDLL(F.LIB_PATH)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_version_and_defaults(F):
    assert F.fftpl_version() == 100
    o = F.fftpl_default_options()
    assert o.target_density == 1.0 and o.dw_ref == 3.5e5 and abs(o.alpha_max0_bins - 0.044) < 1e-15
    assert o.tau_stop == 0.1 and o.solve_path == F.FFTPL_SOLVE_FFT


def _tiny():
    import synth
    return synth.make_instance("tiny")


def _create(F, inst, **kw):
    args = dict(region=inst.region, n=inst.n, w=inst.w, h=inst.h, m_mov=inst.m_mov,
                fix_x=inst.fix_x, fix_y=inst.fix_y, net_ptr=inst.net_ptr, pin_cell=inst.pin_cell,
                pin_dx=inst.pin_dx, pin_dy=inst.pin_dy)
    opts = kw.pop("options", None)
    args.update(kw)
    return F.fftpl_create(options=opts, stream=0, **args)


@pytest.mark.parametrize("change,needle", [
    (dict(n=48), "power of two"),
    (dict(n=8), "power of two"),
    (dict(n=8192), "power of two"),
    (dict(region=(0.0, 0.0, 100.1, 100.1)), "exact in float32"),
    (dict(region=(0.0, 0.0, -5.0, 10.0)), "x1 > x0"),
])
def test_invalid_instances_rejected(F, change, needle):
    inst = _tiny()
    with pytest.raises(F.FFTPLError) as ei:
        _create(F, inst, **change)
    assert ei.value.status == F.FFTPL_EINVAL
    assert needle in str(ei.value)
    assert needle in F.fftpl_last_error(None)


def test_invalid_arrays_rejected(F):
    inst = _tiny()
    bad = inst.pin_cell.copy(); bad[3] = inst.m_mov + 5
    with pytest.raises(F.FFTPLError, match="pin_cell out of range"):
        _create(F, inst, pin_cell=bad)
    w = inst.w.copy(); w[0] = -1.0
    with pytest.raises(F.FFTPLError, match="sizes must be finite"):
        _create(F, inst, w=w)
    w = inst.w.copy(); w[1] = np.nan
    with pytest.raises(F.FFTPLError, match="sizes must be finite"):
        _create(F, inst, w=w)
    npn = inst.net_ptr.copy(); npn[5] = npn[6] + 1
    with pytest.raises(F.FFTPLError, match="non-decreasing"):
        _create(F, inst, net_ptr=npn)
    dx = inst.pin_dx.copy(); dx[0] = np.inf
    with pytest.raises(F.FFTPLError, match="offsets must be finite"):
        _create(F, inst, pin_dx=dx)
    o = F.fftpl_default_options(target_density=0.0)
    with pytest.raises(F.FFTPLError, match="target_density"):
        _create(F, inst, options=o)


def test_null_handle_calls_are_safe(F):
    F.fftpl_destroy(None)
    assert F.fftpl_launch_count(None) == 0
    assert F.fftpl_device_bytes(None) == 0
    assert F.lib().fftpl_check(None) == F.FFTPL_EINVAL
    assert F.lib().fftpl_debug_transpose_stores(None, 1) == F.FFTPL_EINVAL


def test_tensor_core_path_validation(F):
    """The tensor-core solve path needs n >= 128 (128-row tiles); unknown
    paths are rejected; both before any device work."""
    inst = _tiny()          # n = 64
    o = F.fftpl_default_options(solve_path=F.FFTPL_SOLVE_TC_BF16X3)
    with pytest.raises(F.FFTPLError) as ei:
        _create(F, inst, options=o)
    assert ei.value.status == F.FFTPL_EINVAL and "n >= 128" in str(ei.value)
    o = F.fftpl_default_options(solve_path=7)
    with pytest.raises(F.FFTPLError, match="unknown solve_path"):
        _create(F, inst, options=o)


@pytest.mark.parametrize("M,N,K,nsplit", [(100, 128, 64, 3), (128, 128, 96, 3),
                                          (128, 0, 64, 3), (128, 128, 64, 2)])
def test_debug_tc_gemm_validation(F, M, N, K, nsplit):
    """Shapes off the 128 x 128 x 64 tiling, or a bad split, return EINVAL on
    the host (the pointers are never dereferenced)."""
    p = ctypes.c_void_p(1 << 20)
    st = F.lib().fftpl_debug_tc_gemm(p, p, p, p, M, N, K, p, nsplit, 0, p, None)
    assert st == F.FFTPL_EINVAL
    assert "fftpl_debug_tc_gemm" in F.fftpl_last_error(None)


@pytest.mark.parametrize("field,value,needle", [
    ("wirelength", 5, "unknown wirelength model"),
    ("helmholtz_eps", -1e-3, "helmholtz_eps"),
    ("helmholtz_eps", float("nan"), "helmholtz_eps"),
])
def test_variant_options_validated(F, field, value, needle):
    """Model-variant options are checked on the host before device work."""
    o = F.fftpl_default_options(**{field: value})
    with pytest.raises(F.FFTPLError) as ei:
        _create(F, _tiny(), options=o)
    assert ei.value.status == F.FFTPL_EINVAL and needle in str(ei.value)


def test_options_struct_layout(F):
    """The options struct keeps its size (88 bytes) with the variant fields."""
    assert ctypes.sizeof(F.fftpl_options) == 88
    o = F.fftpl_default_options()
    assert o.wirelength == F.FFTPL_WL_WA and o.helmholtz_eps == 0.0


def test_noalloc_validates_before_device_work(F):
    """fftpl_solve_noalloc refuses bad sizes, misaligned maps and bad region
    sizes on the host, before any CUDA call (fake device addresses are never
    dereferenced)."""
    lib = F.lib()
    good, odd = 0x10000, 0x10004
    def call(n, rho=good, Lx=1.0):
        return lib.fftpl_solve_noalloc(ctypes.c_void_p(rho), n, Lx, 1.0, ctypes.c_void_p(good),
                                       ctypes.c_void_p(good), ctypes.c_void_p(good), None, None)
    for n in (8, 1000, 2048, 0, -64):
        assert call(n) == F.FFTPL_EINVAL
    assert call(64, rho=odd) == F.FFTPL_EINVAL
    assert b"aligned" in lib.fftpl_last_error(None)
    assert call(64, Lx=float("nan")) == F.FFTPL_EINVAL
    assert call(64, rho=0) == F.FFTPL_EINVAL
