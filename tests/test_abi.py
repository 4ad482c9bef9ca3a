"""CPU checks of the C ABI: libsrhd.so builds for sm_103a, loads, exports
every entry point that include/srhd.h declares, and its host-side argument
validation works without a GPU (no compute call is made here)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "srhd.h")


def _declared():
    src = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:srhd_status|const char\*)\s+(srhd_\w+)\(", src, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2012_11130_gb300 import build, _native
    path = build.build()
    return _native.load(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("srhd_prim2con", "srhd_con2pri", "srhd_flux_patches", "srhd_advance_patches",
              "srhd_cfl_dt", "srhd_create", "srhd_destroy"):
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    from paper_2012_11130_gb300 import _native
    names = _declared()
    assert sorted(_native.EXPORTS) == names
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True).stdout
    exported = set(re.findall(r" T (srhd_\w+)$", out, re.M))
    assert set(names) <= exported


def test_library_is_built_for_sm103a(lib):
    out = subprocess.run(["cuobjdump", "--list-elf", lib._name], capture_output=True, text=True)
    if out.returncode != 0:
        pytest.skip("cuobjdump unavailable")
    assert "sm_103a" in out.stdout


def test_host_side_validation(lib):
    from paper_2012_11130_gb300 import _native as N
    p = N.Params()
    assert lib.srhd_default_params(ctypes.byref(p)) == N.SRHD_OK
    assert (p.cfl, p.theta, p.retry_factor, p.theta_floor) == (0.5, 1.5, 0.75, 1e-2)
    assert (p.riemann, p.cfl_mode, p.ndim, p.newton_max_iter) == (N.SRHD_HLLC, 0, 3, 0)
    assert lib.srhd_default_params(None) == N.SRHD_ERR_ARG
    # every entry point rejects a NULL context before touching the device
    vp = ctypes.c_void_p
    assert lib.srhd_prim2con(None, 0, vp(1), vp(1), 1, 1, None) == N.SRHD_ERR_ARG
    assert lib.srhd_con2pri(None, 0, vp(1), vp(1), 1, 1, None, None) == N.SRHD_ERR_ARG
    assert lib.srhd_flux_patches(None, 0, vp(1), vp(1), 1, vp(1), None, None) == N.SRHD_ERR_ARG
    assert lib.srhd_advance_patches(None, 0, vp(1), vp(1), None, 1, vp(1), None, None, None,
                                    None) == N.SRHD_ERR_ARG
    assert lib.srhd_cfl_dt(None, 0, vp(1), 1, 0.1, vp(1), None) == N.SRHD_ERR_ARG
    bc = (ctypes.c_int32 * 3)(0, 0, 0)
    dn = ctypes.c_double()
    assert lib.srhd_advance_uniform(None, 0, vp(1), 1, 1, 1, bc, 0, 1, vp(1), None, vp(1), None,
                                    None, None) == N.SRHD_ERR_ARG
    assert lib.srhd_advance_uniform_host(None, 0, vp(1), vp(1), 1, 1, 1, bc, 1e-3, 0.1,
                                         ctypes.byref(dn), None, 8, None) == N.SRHD_ERR_ARG
    assert lib.srhd_advance_amr(None, 0, vp(1), vp(1), vp(1), vp(1), 1, 0.0, None, 0, vp(1),
                                None, 1, vp(1), None, None, None, None) == N.SRHD_ERR_ARG
    assert lib.srhd_fill_ghosts_uniform_range(None, 0, vp(1), vp(1), 1, 1, 1, bc, 0, 1,
                                              None) == N.SRHD_ERR_ARG
    assert b"ctx is NULL" in lib.srhd_last_error()
    assert lib.srhd_destroy(None) == N.SRHD_OK
    # invalid parameters are refused at creation
    h = ctypes.c_void_p()
    bad = N.Params()
    lib.srhd_default_params(ctypes.byref(bad))
    bad.ndim = 4
    assert lib.srhd_create(ctypes.byref(h), ctypes.byref(bad)) == N.SRHD_ERR_ARG
    assert b"ndim" in lib.srhd_last_error()
    assert not h.value


def test_binding_arity_matches_header(lib):
    # every declaration's parameter count equals the ctypes argtypes length
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    decls = re.findall(r"^(?:srhd_status|const char\*)\s+(srhd_\w+)\(([^;]*?)\);", src, re.M | re.S)
    assert decls
    for name, params in decls:
        params = params.strip()
        n = 0 if params in ("", "void") else params.count(",") + 1
        argtypes = getattr(lib, name).argtypes
        assert argtypes is not None and len(argtypes) == n, (name, n, argtypes)
