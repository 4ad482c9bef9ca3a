"""ctypes binding of the FP64 CPU oracle (``srhd_oracle.cpp``).

TEST INFRASTRUCTURE ONLY: a plain, slow restatement of the SRHD scheme of
arXiv 2012.11130 used to check the CUDA library. Only ``tests/``,
``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may
import this module. The product package never imports it.

Every array is float64 and C-contiguous. Layouts follow the library:
primitive W = (rho, U^x, U^y, U^z, p) and conserved U = (D, M^x, M^y, M^z,
Etilde) as structure-of-arrays [5][n]; grids as [5][nz][ny][nx] (x fastest).
Units c = m = k_B = 1; T = p / rho.

Functions whose parity is pinned, and by which test, are listed in the
repository's design notes; none here is "parity unpinned".
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# ORACLE_SRC / ORACLE_LIB override the source and library paths; the
# mutation test uses them to build deliberately broken copies of the oracle.
_SRC = os.environ.get("ORACLE_SRC", os.path.join(_HERE, "srhd_oracle.cpp"))
_LIB = os.environ.get("ORACLE_LIB", os.path.join(_HERE, "liboracle.so"))
_lock = threading.Lock()
_lib = None

# con2pri status codes
OK, UNPHYSICAL, NOCONV = 0, 1, 2
# block-advance status codes
BLK_OK, BLK_UNPHYSICAL, BLK_BAD_INPUT, BLK_NOCONV = 0, 1, 2, 4

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int32)
_up = ctypes.POINTER(ctypes.c_uint64)


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction) if it is stale."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
             "-shared", "-o", tmp, _SRC])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
            for name in ("or_htilde_of_T", "or_T_of_htilde", "or_dT_dhtilde", "or_cs2_of_T"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d]
            for name in ("or_f_of_htilde", "or_df_dhtilde", "or_newton_guess", "or_htilde_bisect",
                         "or_rapidity_integral"):
                getattr(L, name).restype = d
                getattr(L, name).argtypes = [d, d]
            L.or_set_eos.restype = i32
            L.or_set_eos.argtypes = [i32, d]
            L.or_limited_slope.restype = d
            L.or_limited_slope.argtypes = [d, d, d]
            L.or_prim2con.restype = None
            L.or_prim2con.argtypes = [_dp, _dp, i64, _ip, i32]
            L.or_con2pri.restype = None
            L.or_con2pri.argtypes = [_dp, _dp, i64, _ip, _ip, _dp, _dp, i32]
            L.or_phys_flux.restype = None
            L.or_phys_flux.argtypes = [i32, _dp, _dp, _dp, i32]
            L.or_char_speeds.restype = None
            L.or_char_speeds.argtypes = [i32, _dp, _dp, _dp]
            L.or_riemann_flux.restype = i32
            L.or_riemann_flux.argtypes = [i32, i32, _dp, _dp, _dp, _dp, _dp, i32]
            L.or_smax.restype = d
            L.or_smax.argtypes = [_dp, i32]
            L.or_advance_block.restype = i32
            L.or_advance_block.argtypes = [_dp, _dp, _dp, i32, i32, i32, i32, i32, i32, d, d, d,
                                           d, d, i32, _ip, i32]
            L.or_advance_patches.restype = None
            L.or_advance_patches.argtypes = [_dp, _dp, i64, _dp, d, d, d, i32, _ip, _ip, _dp, i32]
            L.or_advance_block_vl.restype = i32
            L.or_advance_block_vl.argtypes = L.or_advance_block.argtypes
            L.or_advance_patches_vl.restype = None
            L.or_advance_patches_vl.argtypes = L.or_advance_patches.argtypes
            L.or_cfl_dt.restype = d
            L.or_cfl_dt.argtypes = [_dp, i64, d, d, i32, i32, i32]
            L.or_count_advance_block.restype = None
            L.or_count_advance_block.argtypes = [_dp, i32, i32, i32, i32, i32, i32, d, d, d, i32,
                                                 _up]
            L.or_count_advance_block_vl.restype = None
            L.or_count_advance_block_vl.argtypes = L.or_count_advance_block.argtypes
            L.or_count_cfl.restype = None
            L.or_count_cfl.argtypes = [_dp, i64, i32, _up]
            L.or_exact_riemann.restype = None
            L.or_exact_riemann.argtypes = [d, d, d, d, d, d, d, d, _dp, i64, _dp, _dp, _dp, _dp]
            _lib = L
    return _lib


def _p(a, t=_dp):
    return a.ctypes.data_as(t) if a is not None else None


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


# --- Section 2.2: TM equation of state ------------------------------------
# --- equation of state selection (Section 2.2) ---------------------------------
EOS_TM, EOS_POLYTROPIC = 0, 1


def set_eos(kind=EOS_TM, gamma=5.0 / 3.0):
    """Select the EoS of every following oracle call on this thread: the
    Taub-Mathews EoS (default) or the polytropic h = 1 + Gamma/(Gamma-1) T
    with 1 < Gamma <= 5/3."""
    if lib().or_set_eos(int(kind), float(gamma)) != 0:
        raise ValueError(f"invalid EoS selection kind={kind} gamma={gamma}")


@contextlib.contextmanager
def eos(kind=EOS_TM, gamma=5.0 / 3.0):
    """Context in which the oracle uses the given EoS (restores TM after)."""
    set_eos(kind, gamma)
    try:
        yield
    finally:
        set_eos(EOS_TM)


def htilde_of_T(T):
    """Eq. (T_to_HTilde)."""
    return np.vectorize(lib().or_htilde_of_T, otypes=[float])(T)


def T_of_htilde(ht):
    """Eq. (T of h)."""
    return np.vectorize(lib().or_T_of_htilde, otypes=[float])(ht)


def dT_dhtilde(ht):
    """Eq. (dT_dh)."""
    return np.vectorize(lib().or_dT_dhtilde, otypes=[float])(ht)


def cs2_of_T(T):
    """Eq. (sound_speed), squared."""
    return np.vectorize(lib().or_cs2_of_T, otypes=[float])(T)


def f_of_htilde(ht, m2):
    """Eq. (transcendental equation), right-hand side f(htilde; m^2)."""
    return np.vectorize(lib().or_f_of_htilde, otypes=[float])(ht, m2)


def df_dhtilde(ht, m2):
    """Appendix A, df/dhtilde."""
    return np.vectorize(lib().or_df_dhtilde, otypes=[float])(ht, m2)


def newton_guess(A, m2):
    """Appendix A, initial guess (hot / cold with the Eq. ColdHot threshold)."""
    return np.vectorize(lib().or_newton_guess, otypes=[float])(A, m2)


def htilde_bisect(A, m2):
    """Brute-force root of f(htilde) = A by bisection to one ulp."""
    return np.vectorize(lib().or_htilde_bisect, otypes=[float])(A, m2)


def limited_slope(dl, dr, theta):
    """Hybrid van Leer / generalised minmod slope."""
    return np.vectorize(lib().or_limited_slope, otypes=[float])(dl, dr, theta)


# --- Section 2.3: conversions -----------------------------------------------
# scheme 0: the paper's new scheme (reduced energy Etilde); scheme 1: the
# "original" scheme it compares against (total energy E with flux M).
NEW, ORIGINAL = 0, 1


def prim2con(prim, scheme=NEW):
    """prim [5][n] -> (cons [5][n], status [n])."""
    prim = _f64(prim)
    n = prim.shape[1]
    cons = np.empty_like(prim)
    st = np.empty(n, np.int32)
    lib().or_prim2con(_p(prim), _p(cons), n, _p(st, _ip), scheme)
    return cons, st


def con2pri(cons, scheme=NEW):
    """cons [5][n] -> dict(prim, status, iters, htilde, A)."""
    cons = _f64(cons)
    n = cons.shape[1]
    prim = np.empty_like(cons)
    st = np.empty(n, np.int32)
    it = np.empty(n, np.int32)
    ht = np.empty(n)
    A = np.empty(n)
    lib().or_con2pri(_p(cons), _p(prim), n, _p(st, _ip), _p(it, _ip), _p(ht), _p(A), scheme)
    return dict(prim=prim, status=st, iters=it, htilde=ht, A=A)


# --- Section 3: scheme pieces ---------------------------------------------
def phys_flux(d, W, scheme=NEW):
    W = _f64(W)
    U, st = prim2con(W.reshape(5, 1), scheme)
    F = np.empty(5)
    lib().or_phys_flux(d, _p(W), _p(_f64(U[:, 0])), _p(F), scheme)
    return F


def char_speeds(d, W):
    W = _f64(W)
    lm, lp = ctypes.c_double(), ctypes.c_double()
    lib().or_char_speeds(d, _p(W), ctypes.byref(lm), ctypes.byref(lp))
    return lm.value, lp.value


def riemann_flux(d, WL, WR, solver=0, UL=None, UR=None, scheme=NEW):
    """Riemann flux across a face normal to d (0 = HLLC, 1 = HLLE).

    Returns (F[5], fell_back_to_hlle)."""
    WL, WR = _f64(WL), _f64(WR)
    if UL is None:
        UL = prim2con(WL.reshape(5, 1), scheme)[0][:, 0]
    if UR is None:
        UR = prim2con(WR.reshape(5, 1), scheme)[0][:, 0]
    UL, UR = _f64(UL), _f64(UR)
    F = np.empty(5)
    fb = lib().or_riemann_flux(d, solver, _p(WL), _p(UL), _p(WR), _p(UR), _p(F), scheme)
    return F, fb


def smax(W, ndim=3):
    return lib().or_smax(_p(_f64(W)), ndim)


DEFAULT_THETA = 1.5
RETRY_FACTOR = 0.75
THETA_FLOOR = 1e-2


def advance_block(cons, n, act, dt, dh, theta=DEFAULT_THETA, riemann=0, want_flux=False,
                  retry_factor=RETRY_FACTOR, theta_floor=THETA_FLOOR, scheme=NEW):
    """One MUSCL-Hancock step of a block with ghosts.

    cons: [5][Nz][Ny][Nx] with N_d = n_d + 4 on active dims, n_d otherwise.
    Returns dict(out [5][nz][ny][nx], status, retries, flux (optional))."""
    cons = _f64(cons)
    nx, ny, nz = n
    out = np.empty((5, nz, ny, nx))
    flux = None
    if want_flux:
        nf = sum(((nx * ny * nz) // n[d]) * (n[d] + 1) for d in range(3) if act[d])
        flux = np.empty(5 * nf)
    r = np.zeros(1, np.int32)
    st = lib().or_advance_block(_p(cons), _p(out), _p(flux), nx, ny, nz, int(act[0]),
                                int(act[1]), int(act[2]), dt, dh, theta, retry_factor,
                                theta_floor, riemann, _p(r, _ip), scheme)
    return dict(out=out, status=st, retries=int(r[0]), flux=flux)


def advance_patches(cons, dt_dh, theta=DEFAULT_THETA, riemann=0, want_flux=False, scheme=NEW):
    """Batched step of independent 8^3 patches with 2-cell ghosts.

    cons [np][5][12][12][12] -> dict(out [np][5][8][8][8], status, retries,
    flux [np][3][5][9*8*8] if requested)."""
    cons = _f64(cons)
    npatch = cons.shape[0]
    out = np.empty((npatch, 5, 8, 8, 8))
    st = np.empty(npatch, np.int32)
    rt = np.empty(npatch, np.int32)
    flux = np.empty((npatch, 3, 5, 576)) if want_flux else None
    dt_dh = _f64(dt_dh).reshape(npatch, 2)
    lib().or_advance_patches(_p(cons), _p(out), npatch, _p(dt_dh), theta, RETRY_FACTOR,
                             THETA_FLOOR, riemann, _p(st, _ip), _p(rt, _ip), _p(flux), scheme)
    return dict(out=out, status=st, retries=rt, flux=flux)


def advance_block_vl(cons, n, act, dt, dh, theta=DEFAULT_THETA, riemann=0, want_flux=False,
                     retry_factor=RETRY_FACTOR, theta_floor=THETA_FLOOR, scheme=NEW):
    """One VL (predictor-corrector) step of a block with 3 ghost cells on
    active dims: cons [5][Nz][Ny][Nx], N_d = n_d + 6 on active dims."""
    cons = _f64(cons)
    nx, ny, nz = n
    out = np.empty((5, nz, ny, nx))
    flux = None
    if want_flux:
        nf = sum(((nx * ny * nz) // n[d]) * (n[d] + 1) for d in range(3) if act[d])
        flux = np.empty(5 * nf)
    r = np.zeros(1, np.int32)
    st = lib().or_advance_block_vl(_p(cons), _p(out), _p(flux), nx, ny, nz, int(act[0]),
                                   int(act[1]), int(act[2]), dt, dh, theta, retry_factor,
                                   theta_floor, riemann, _p(r, _ip), scheme)
    return dict(out=out, status=st, retries=int(r[0]), flux=flux)


def advance_patches_vl(cons, dt_dh, theta=DEFAULT_THETA, riemann=0, want_flux=False,
                       scheme=NEW):
    """Batched VL step of independent 8^3 patches with 3-cell ghosts:
    cons [np][5][14][14][14] -> dict(out [np][5][8][8][8], status, retries,
    flux [np][3][5][576] if requested)."""
    cons = _f64(cons)
    npatch = cons.shape[0]
    out = np.empty((npatch, 5, 8, 8, 8))
    st = np.empty(npatch, np.int32)
    rt = np.empty(npatch, np.int32)
    flux = np.empty((npatch, 3, 5, 576)) if want_flux else None
    dt_dh = _f64(dt_dh).reshape(npatch, 2)
    lib().or_advance_patches_vl(_p(cons), _p(out), npatch, _p(dt_dh), theta, RETRY_FACTOR,
                                THETA_FLOOR, riemann, _p(st, _ip), _p(rt, _ip), _p(flux), scheme)
    return dict(out=out, status=st, retries=rt, flux=flux)


def cfl_dt(cons, dh, cfl=0.5, ndim=3, cfl_mode=0, scheme=NEW):
    """Eq. (time_step_sound_speed): min over cells cons [5][n]."""
    cons = _f64(cons).reshape(5, -1)
    return lib().or_cfl_dt(_p(cons), cons.shape[1], dh, cfl, ndim, cfl_mode, scheme)


def count_advance_block(cons, n, act, dt, dh, theta=DEFAULT_THETA, riemann=0):
    """Operation tally (add, mul, div, sqrt) of one block advance."""
    cons = _f64(cons)
    c = np.zeros(4, np.uint64)
    lib().or_count_advance_block(_p(cons), n[0], n[1], n[2], int(act[0]), int(act[1]),
                                 int(act[2]), dt, dh, theta, riemann, _p(c, _up))
    return dict(add=int(c[0]), mul=int(c[1]), div=int(c[2]), sqrt=int(c[3]))


def count_advance_block_vl(cons, n, act, dt, dh, theta=DEFAULT_THETA, riemann=0):
    """Operation tally of one VL block advance (3 ghost cells on active dims)."""
    cons = _f64(cons)
    c = np.zeros(4, np.uint64)
    lib().or_count_advance_block_vl(_p(cons), n[0], n[1], n[2], int(act[0]), int(act[1]),
                                    int(act[2]), dt, dh, theta, riemann, _p(c, _up))
    return dict(add=int(c[0]), mul=int(c[1]), div=int(c[2]), sqrt=int(c[3]))


def count_cfl(cons, ndim=3):
    cons = _f64(cons).reshape(5, -1)
    c = np.zeros(4, np.uint64)
    lib().or_count_cfl(_p(cons), cons.shape[1], ndim, _p(c, _up))
    return dict(add=int(c[0]), mul=int(c[1]), div=int(c[2]), sqrt=int(c[3]))


# --- Appendix C: exact Riemann solution -------------------------------------
def exact_riemann(left, right, x0, t, x):
    """left/right = (rho, U, p); returns (rho, U, p, info dict) at x."""
    x = _f64(x)
    n = x.size
    rho, U, p = np.empty(n), np.empty(n), np.empty(n)
    info = np.empty(10)
    lib().or_exact_riemann(float(left[0]), float(left[1]), float(left[2]), float(right[0]),
                           float(right[1]), float(right[2]), x0, t, _p(x), n, _p(rho), _p(U),
                           _p(p), _p(info))
    keys = ["pstar", "U_CL", "U_CR", "rho_CL", "rho_CR", "shock_L", "shock_R", "Ushock_L",
            "Ushock_R", "T_CL"]
    return rho, U, p, dict(zip(keys, info.tolist()))


def rapidity_integral(T1, T2):
    return lib().or_rapidity_integral(T1, T2)


# --- whole-domain driver (plain Python loop over oracle steps) -------------
def fill_ghosts(interior, act, bc, width=2):
    """Pad [5][nz][ny][nx] with `width` ghost cells on active dims (2 for
    MUSCL-Hancock, 3 for VL).

    bc: 'periodic' (wrap) or 'outflow' (zero-gradient copy of the edge cell)."""
    mode = "wrap" if bc == "periodic" else "edge"
    pads = [(0, 0)] + [((width, width) if act[d] else (0, 0)) for d in (2, 1, 0)]
    return np.pad(interior, pads, mode=mode)


def evolve(cons, act, dh, t_end, bc, cfl=0.5, theta=DEFAULT_THETA, riemann=0, max_steps=10**7,
           scheme=NEW, integrator="mh"):
    """Advance the whole domain to t_end: each step takes the CFL time step
    of the current state (clipped to reach t_end exactly), fills ghosts and
    applies one block step (integrator "mh": MUSCL-Hancock, "vl": VL).
    Returns dict(cons, t, steps, retries)."""
    cons = _f64(cons).copy()
    nz, ny, nx = cons.shape[1:]
    n = (nx, ny, nz)
    ndim = int(sum(bool(a) for a in act))
    t = 0.0
    steps = 0
    retries = 0
    while t < t_end and steps < max_steps:
        dt = cfl_dt(cons, dh, cfl=cfl, ndim=ndim, scheme=scheme)
        if not np.isfinite(dt):
            raise RuntimeError("unphysical state in CFL")
        if t + dt > t_end:
            dt = t_end - t
        if integrator == "vl":
            r = advance_block_vl(fill_ghosts(cons, act, bc, 3), n, act, dt, dh, theta=theta,
                                 riemann=riemann, scheme=scheme)
        else:
            r = advance_block(fill_ghosts(cons, act, bc), n, act, dt, dh, theta=theta,
                              riemann=riemann, scheme=scheme)
        if r["status"] not in (BLK_OK, BLK_NOCONV):
            raise RuntimeError(f"block step failed with status {r['status']}")
        retries += r["retries"]
        cons = r["out"]
        t += dt
        steps += 1
    return dict(cons=cons, t=t, steps=steps, retries=retries)
