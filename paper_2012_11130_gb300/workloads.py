"""Seeded synthetic inputs shaped like the test problems of arXiv 2012.11130.

This module only draws primitive states (rho, U^x, U^y, U^z, p) and moves
arrays between layouts; it holds none of the method's arithmetic (no EoS, no
conversion), so that the CUDA path and the CPU oracle can both consume its
output. Arrays are float64 numpy arrays (or torch tensors where noted).

Workloads (units c = m = k_B = 1):
  * stress batch: rho log-uniform in [1e-6, 1e2], T = p/rho log-uniform in
    [1e-8, 1e4], Lorentz factor log-uniform in [1, 1e6], direction uniform on
    the sphere; U = sqrt(gamma^2 - 1) n.
  * shock tube: 1024 cells on [0, 1], (rho, v, p) = (1, 0, 1e3) | (1, 0, 1e-2)
    at x = 0.5.
  * smooth advection: [0, 1]^3 periodic, rho = 1 + 0.5 sin(2 pi (x+y+z)),
    p = 1, U = sqrt(99/3) along each axis (gamma = 10 along the diagonal).
  * rough patches: independent 12^3 ghosted patches of uncorrelated cells
    (rho, T log-uniform over +-spread decades, gamma up to 10^1.5), which
    drive the limiter retry of Section 3.3.
"""
from __future__ import annotations

import numpy as np

PATCH = 8
GHOST = 2
GP = PATCH + 2 * GHOST


def stress_batch_prims(n: int, seed: int = 12345, rho_range=(-6.0, 2.0), T_range=(-8.0, 4.0),
                       lg_gamma_range=(0.0, 6.0)) -> np.ndarray:
    rng = np.random.default_rng(seed)
    rho = 10.0 ** rng.uniform(*rho_range, n)
    T = 10.0 ** rng.uniform(*T_range, n)
    gam = 10.0 ** rng.uniform(*lg_gamma_range, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    U = np.sqrt(gam * gam - 1.0) * d
    return np.vstack([rho, U, rho * T])


def stress_batch_prims_torch(n: int, seed: int = 12345, device="cuda"):
    """Same distribution drawn on the device with torch (for large n)."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    u = lambda lo, hi: lo + (hi - lo) * torch.rand(n, generator=g, device=device,
                                                   dtype=torch.float64)
    rho = 10.0 ** u(-6.0, 2.0)
    T = 10.0 ** u(-8.0, 4.0)
    gam = 10.0 ** u(0.0, 6.0)
    d = torch.randn(3, n, generator=g, device=device, dtype=torch.float64)
    d = d / torch.linalg.vector_norm(d, dim=0)
    U = torch.sqrt(gam * gam - 1.0) * d
    return torch.cat([rho[None], U, (rho * T)[None]], 0)


def shock_tube_prims(n: int = 1024, x0: float = 0.5, left=(1.0, 0.0, 1e3),
                     right=(1.0, 0.0, 1e-2)) -> tuple[np.ndarray, np.ndarray]:
    """Cell-centred 1-D primitive field [5][n] on [0, 1] and the centres."""
    x = (np.arange(n) + 0.5) / n
    L = x < x0
    W = np.zeros((5, n))
    W[0] = np.where(L, left[0], right[0])
    W[1] = np.where(L, left[1], right[1])
    W[4] = np.where(L, left[2], right[2])
    return W, x


def advection_prims(n: int, amp: float = 0.5, Uaxis: float = float(np.sqrt(99.0 / 3.0)),
                    p: float = 1.0, t: float = 0.0) -> np.ndarray:
    """[5][n][n][n] primitive field of the diagonal sine wave (z, y, x order)
    translated by the bulk three-velocity times t."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    v = Uaxis / np.sqrt(1.0 + 3.0 * Uaxis * Uaxis)  # per-axis three-velocity
    rho = 1.0 + amp * np.sin(2.0 * np.pi * ((x - v * t) + (y - v * t) + (z - v * t)))
    W = np.empty((5, n, n, n))
    W[0] = rho
    W[1:4] = Uaxis
    W[4] = p
    return W


def advection_ghosted_patch_prims(n: int, patches, amp: float = 0.5,
                                  Uaxis: float = float(np.sqrt(99.0 / 3.0)),
                                  p: float = 1.0) -> np.ndarray:
    """[m][5][12][12][12] primitive values of the periodic diagonal sine wave
    on the ghosted patches with the given indices (patch (ix,iy,iz) at
    (iz*npy + iy)*npx + ix, npx = npy = npz = n/8), ghosts wrapped."""
    patches = np.asarray(patches)
    npx = n // PATCH
    ix, iy, iz = patches % npx, (patches // npx) % npx, patches // (npx * npx)
    g = np.arange(GP) - GHOST
    cx = ((ix[:, None] * PATCH + g[None, :]) % n + 0.5) / n
    cy = ((iy[:, None] * PATCH + g[None, :]) % n + 0.5) / n
    cz = ((iz[:, None] * PATCH + g[None, :]) % n + 0.5) / n
    phase = cz[:, :, None, None] + cy[:, None, :, None] + cx[:, None, None, :]
    W = np.empty((patches.size, 5, GP, GP, GP))
    W[:, 0] = 1.0 + amp * np.sin(2.0 * np.pi * phase)
    W[:, 1:4] = Uaxis
    W[:, 4] = p
    return W


def rough_patch_prims(npatch: int, seed: int = 0, spread: float = 1.0,
                      lg_gamma_max: float = 1.5) -> np.ndarray:
    """[np][5][12][12][12] uncorrelated ghosted patches."""
    rng = np.random.default_rng(seed)
    n = npatch * GP ** 3
    rho = 10.0 ** rng.uniform(-spread, spread, n)
    T = 10.0 ** rng.uniform(-spread, spread, n)
    gam = 10.0 ** rng.uniform(0.0, lg_gamma_max, n)
    d = rng.normal(size=(3, n))
    d /= np.linalg.norm(d, axis=0)
    U = np.sqrt(gam * gam - 1.0) * d
    W = np.vstack([rho, U, rho * T])
    return W.reshape(5, npatch, GP, GP, GP).transpose(1, 0, 2, 3, 4).copy()


def smooth_patch_prims(npatch: int, seed: int = 0, amp: float = 0.3,
                       Umax: float = 0.5) -> np.ndarray:
    """[np][5][12][12][12] patches of smooth random waves (no retry expected)."""
    rng = np.random.default_rng(seed)
    c = np.arange(GP) / GP
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    out = np.empty((npatch, 5, GP, GP, GP))
    for q in range(npatch):
        ph = rng.uniform(0, 2 * np.pi, 8)
        k = rng.integers(1, 3, 6)
        out[q, 0] = 1.0 + amp * np.sin(2 * np.pi * (k[0] * x + k[1] * y) + ph[0])
        out[q, 4] = 1.0 + amp * np.sin(2 * np.pi * (k[2] * y - z) + ph[1])
        out[q, 1] = Umax * np.sin(2 * np.pi * (x + k[3] * z) + ph[2])
        out[q, 2] = Umax * np.cos(2 * np.pi * (k[4] * x - y) + ph[3])
        out[q, 3] = Umax * np.sin(2 * np.pi * (k[5] * z + y) + ph[4])
    return out


# ---- layouts (no arithmetic) -------------------------------------------------
def patchify(field: np.ndarray) -> np.ndarray:
    """[5][nz][ny][nx] -> [np][5][8][8][8], patch (ix,iy,iz) at (iz*npy+iy)*npx+ix."""
    _, nz, ny, nx = field.shape
    pz, py, px = nz // PATCH, ny // PATCH, nx // PATCH
    f = field.reshape(5, pz, PATCH, py, PATCH, px, PATCH)
    return f.transpose(1, 3, 5, 0, 2, 4, 6).reshape(pz * py * px, 5, PATCH, PATCH, PATCH).copy()


def unpatchify(patches: np.ndarray, npx: int, npy: int, npz: int) -> np.ndarray:
    f = patches.reshape(npz, npy, npx, 5, PATCH, PATCH, PATCH)
    return f.transpose(3, 0, 4, 1, 5, 2, 6).reshape(5, npz * PATCH, npy * PATCH, npx * PATCH).copy()


def ghosted_patches(field: np.ndarray, bc=("periodic", "periodic", "periodic")) -> np.ndarray:
    """[5][nz][ny][nx] -> [np][5][12][12][12] with 2 ghost cells from the
    neighbouring patches or the boundary (bc per axis x, y, z: 'periodic'
    wraps, 'outflow' copies the edge cell)."""
    mode = {"periodic": "wrap", "outflow": "edge"}
    padded = field
    for ax, b in zip((3, 2, 1), bc):
        pads = [(0, 0)] * 4
        pads[ax] = (GHOST, GHOST)
        padded = np.pad(padded, pads, mode=mode[b])
    _, nz, ny, nx = field.shape
    pz, py, px = nz // PATCH, ny // PATCH, nx // PATCH
    out = np.empty((pz * py * px, 5, GP, GP, GP), dtype=field.dtype)
    q = 0
    for iz in range(pz):
        for iy in range(py):
            for ix in range(px):
                out[q] = padded[:, iz * PATCH:iz * PATCH + GP, iy * PATCH:iy * PATCH + GP,
                                ix * PATCH:ix * PATCH + GP]
                q += 1
    return out
