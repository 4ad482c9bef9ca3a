"""ctypes loader of libsrhd.so with the C signatures of include/srhd.h.

The CUDA library is the only implementation of the fluid update: if it is
missing or fails to load, importing this module raises, and nothing falls
back to another code path.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libsrhd.so")

SRHD_OK, SRHD_ERR_ARG, SRHD_ERR_CUDA = 0, 1, 2
SRHD_FP64, SRHD_MIXED, SRHD_MIXED_CF = 0, 1, 2
SRHD_HLLC, SRHD_HLLE = 0, 1
SRHD_CFL_SIGNAL, SRHD_CFL_LIGHT = 0, 1
SRHD_BC_PERIODIC, SRHD_BC_OUTFLOW = 0, 1
SRHD_SCHEME_REDUCED, SRHD_SCHEME_TOTAL = 0, 1
SRHD_EOS_TM, SRHD_EOS_POLYTROPIC = 0, 1
CELL_OK, CELL_UNPHYSICAL, CELL_NOCONV = 0, 1, 2
PATCH_UNPHYSICAL, PATCH_BAD_INPUT, PATCH_NOCONV, PATCH_STAGE_TIMEOUT = 1, 2, 4, 8

# Every symbol declared in include/srhd.h.
EXPORTS = ("srhd_default_params", "srhd_create", "srhd_destroy", "srhd_last_error",
           "srhd_prim2con", "srhd_con2pri", "srhd_flux_patches", "srhd_advance_patches",
           "srhd_cfl_dt", "srhd_fill_ghosts_uniform", "srhd_cfl_dt_noalloc",
           "srhd_amr_fill_ghosts", "srhd_amr_restrict", "srhd_amr_flux_correct",
           "srhd_advance_patches_vl", "srhd_fill_ghosts_uniform3",
           "srhd_fill_ghosts_uniform_range", "srhd_advance_uniform_host",
           "srhd_advance_uniform", "srhd_advance_amr", "srhd_con2pri_patches",
           "srhd_advance_uniform_prim", "srhd_reciprocal_f64", "srhd_amr_prolong")
SRHD_AMR_COARSE = 1 << 30


class Params(ctypes.Structure):
    _fields_ = [("cfl", ctypes.c_double), ("theta", ctypes.c_double),
                ("retry_factor", ctypes.c_double), ("theta_floor", ctypes.c_double),
                ("riemann", ctypes.c_int32), ("cfl_mode", ctypes.c_int32),
                ("ndim", ctypes.c_int32), ("newton_max_iter", ctypes.c_int32),
                ("patch_variant", ctypes.c_int32), ("scheme", ctypes.c_int32),
                ("eos", ctypes.c_int32), ("gamma", ctypes.c_double)]


class SrhdError(RuntimeError):
    pass


_lib = None


def load(path: str = LIB_PATH):
    """Load libsrhd.so and declare its signatures (raises if absent)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with paper_2012_11130_gb300.build.build()")
    L = ctypes.CDLL(path)
    vp, i64, i32, d = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double
    i32p = ctypes.POINTER(ctypes.c_int32)
    st = ctypes.c_int
    L.srhd_default_params.restype = st
    L.srhd_default_params.argtypes = [ctypes.POINTER(Params)]
    L.srhd_create.restype = st
    L.srhd_create.argtypes = [ctypes.POINTER(vp), ctypes.POINTER(Params)]
    L.srhd_destroy.restype = st
    L.srhd_destroy.argtypes = [vp]
    L.srhd_last_error.restype = ctypes.c_char_p
    L.srhd_last_error.argtypes = []
    L.srhd_prim2con.restype = st
    L.srhd_prim2con.argtypes = [vp, ctypes.c_int, vp, vp, i64, i64, vp]
    L.srhd_con2pri.restype = st
    L.srhd_con2pri.argtypes = [vp, ctypes.c_int, vp, vp, i64, i64, vp, vp]
    L.srhd_flux_patches.restype = st
    L.srhd_flux_patches.argtypes = [vp, ctypes.c_int, vp, vp, i32, vp, vp, vp]
    L.srhd_advance_patches.restype = st
    L.srhd_advance_patches.argtypes = [vp, ctypes.c_int, vp, vp, vp, i32, vp, vp, vp, vp, vp]
    L.srhd_cfl_dt.restype = st
    L.srhd_cfl_dt.argtypes = [vp, ctypes.c_int, vp, i32, d, vp, vp]
    L.srhd_fill_ghosts_uniform.restype = st
    L.srhd_fill_ghosts_uniform.argtypes = [vp, ctypes.c_int, vp, vp, i32, i32, i32, i32p, vp]
    L.srhd_advance_patches_vl.restype = st
    L.srhd_advance_patches_vl.argtypes = L.srhd_advance_patches.argtypes
    L.srhd_fill_ghosts_uniform_range.restype = st
    L.srhd_fill_ghosts_uniform_range.argtypes = [vp, ctypes.c_int, vp, vp, i32, i32, i32, i32p,
                                                 i32, i32, vp]
    L.srhd_advance_uniform.restype = st
    L.srhd_advance_uniform.argtypes = [vp, ctypes.c_int, vp, i32, i32, i32, i32p, i32, i32, vp,
                                       vp, vp, vp, vp, vp]
    L.srhd_con2pri_patches.restype = st
    L.srhd_con2pri_patches.argtypes = [vp, ctypes.c_int, vp, i64, vp, vp]
    L.srhd_advance_uniform_prim.restype = st
    L.srhd_advance_uniform_prim.argtypes = [vp, ctypes.c_int, vp, vp, i32, i32, i32, i32p, i32,
                                            i32, vp, vp, vp, vp, vp, vp, vp]
    L.srhd_reciprocal_f64.restype = st
    L.srhd_reciprocal_f64.argtypes = [vp, vp, i64, vp]
    L.srhd_advance_amr.restype = st
    L.srhd_advance_amr.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, i32, ctypes.c_double, vp,
                                   i32, vp, vp, i32, vp, vp, vp, vp, vp]
    L.srhd_advance_uniform_host.restype = st
    L.srhd_advance_uniform_host.argtypes = [vp, ctypes.c_int, vp, vp, i32, i32, i32, i32p,
                                            ctypes.c_double, ctypes.c_double,
                                            ctypes.POINTER(ctypes.c_double), i32p, i32, vp]
    L.srhd_fill_ghosts_uniform3.restype = st
    L.srhd_fill_ghosts_uniform3.argtypes = L.srhd_fill_ghosts_uniform.argtypes
    L.srhd_cfl_dt_noalloc.restype = st
    L.srhd_cfl_dt_noalloc.argtypes = [ctypes.c_int, vp, i32, d, ctypes.POINTER(Params), vp, vp]
    L.srhd_amr_fill_ghosts.restype = st
    L.srhd_amr_fill_ghosts.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, i32, i32, i32, d, vp,
                                       i32, vp]
    L.srhd_amr_restrict.restype = st
    L.srhd_amr_restrict.argtypes = [vp, ctypes.c_int, vp, vp, i32, i32, vp]
    L.srhd_amr_flux_correct.restype = st
    L.srhd_amr_flux_correct.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, vp, i32, vp, i32, vp,
                                         vp]
    L.srhd_amr_prolong.restype = st
    L.srhd_amr_prolong.argtypes = [vp, ctypes.c_int, vp, vp, vp, i32, i32, d, vp, vp, vp]
    _lib = L
    return L


def check(status: int, what: str) -> None:
    if status != SRHD_OK:
        msg = _lib.srhd_last_error().decode() if _lib is not None else ""
        raise SrhdError(f"{what} failed with status {status}: {msg}")
