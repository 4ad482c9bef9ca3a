"""Shared helpers of the GPU parity tests: the library context, conversions
between numpy and torch, and the tolerance rules.

Tolerance rule (both precisions): a conversion of a cell whose conditioning
kappa = 1 + Mach^2 (Eq. ImprovedRelativeError) is large loses log10(kappa)
digits in any correct implementation, so per-cell relative differences are
allowed up to max(base, 10 kappa eps_A), eps_A the precision of A (eps64, or
about 2^-44 for the compensated float A of mixed_cf), with base = 1e-12 for the FP64 path
and 1e-5 for the mixed path (float storage and arithmetic with the hardware
approximate division and square root, A in double; the observed tail of a
2^18-cell stress batch is 8e-6, i.e. about 64 float ulps).
"""
import numpy as np
import pytest

EPS64 = np.finfo(np.float64).eps
BASE_FP64 = 1e-12
BASE_MIXED = 1e-5
# Relative precision of A in each path: double, double, and the compensated
# float sum of the mixed_cf path (about 4 eps_float^2 of the cancelling terms).
EPS_A = {"fp64": EPS64, "mixed": EPS64, "mixed_cf": 4 * 2.0 ** -46}
BASE = {"fp64": BASE_FP64, "mixed": BASE_MIXED, "mixed_cf": BASE_MIXED}
PRECS = ("fp64", "mixed", "mixed_cf")


def torch_dtype(torch, prec):
    return torch.float64 if prec == "fp64" else torch.float32


def require_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2012_11130_gb300 import build
    build.build()
    from paper_2012_11130_gb300 import srhd
    return torch, srhd


def to_dev(torch, a, dtype):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dtype, device="cuda")


def to_np(t):
    return t.detach().cpu().double().numpy()


def kappa_of_prims(oracle, W):
    """1 + Mach^2 with Mach = |U| / U_s (Eq. MachNumber)."""
    W = np.asarray(W).reshape(5, -1)
    T = W[4] / W[0]
    cs2 = oracle.cs2_of_T(T)
    Us2 = cs2 / (1.0 - cs2)
    return 1.0 + (W[1] ** 2 + W[2] ** 2 + W[3] ** 2) / Us2


def cons_rel_err(a, b):
    """Per-cell relative difference of conserved arrays [5][n]: D and
    Etilde relative to themselves, momentum relative to |M| + Etilde."""
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    e = np.empty_like(a)
    e[0] = np.abs(a[0] - b[0]) / np.abs(b[0])
    sM = np.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2) + np.abs(b[4])
    for k in (1, 2, 3):
        e[k] = np.abs(a[k] - b[k]) / sM
    e[4] = np.abs(a[4] - b[4]) / np.abs(b[4])
    return e.max(axis=0)


def prim_rel_err(a, b):
    """Per-cell relative difference of primitive arrays [5][n]: rho, p
    relative; four-velocity relative to |U| + 1e-300."""
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    e = np.empty_like(a)
    e[0] = np.abs(a[0] - b[0]) / np.abs(b[0])
    sU = np.sqrt(b[1] ** 2 + b[2] ** 2 + b[3] ** 2) + 1e-300
    for k in (1, 2, 3):
        e[k] = np.abs(a[k] - b[k]) / sU
    e[4] = np.abs(a[4] - b[4]) / np.abs(b[4])
    return e.max(axis=0)


def flux_rel_err(a, b):
    """Per-face difference of flux arrays [5][n] relative to the face's
    largest flux component (fluxes can change sign)."""
    a = np.asarray(a).reshape(5, -1)
    b = np.asarray(b).reshape(5, -1)
    s = np.abs(b).max(axis=0) + 1e-300
    return (np.abs(a - b) / s).max(axis=0)
