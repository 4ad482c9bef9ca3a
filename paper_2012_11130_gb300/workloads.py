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
                      lg_gamma_max: float = 1.5, edge: int = GP) -> np.ndarray:
    """[np][5][edge]^3 uncorrelated ghosted patches (edge 12, or 14 for VL)."""
    GP = edge  # noqa: N806
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
                       Umax: float = 0.5, edge: int = GP) -> np.ndarray:
    """[np][5][edge]^3 patches of smooth random waves (no retry expected;
    edge 12, or 14 for the VL integrator's three ghost cells)."""
    GP = edge  # noqa: N806
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


# ---- batched AMR: off-centre relativistic blast wave ---------------------
def blast_prims_at(x, y, z, center=(0.6, 0.5, 0.5), r_shell=0.18, shell=0.01, width=0.002,
                   rho_in=0.05, rho_shell=8.0, rho_amb=1.0, p_in=10.0, p_amb=1e-6,
                   U_shell=4.0, xp=np):
    """Primitive state of a synthetic evolved blast wave (a hot rarefied
    interior, a dense shell moving outward with four-velocity ~U_shell, cold
    ambient gas at rest; tanh transitions of the given width) at points
    (x, y, z); returns [5][...]. xp is the array module (numpy or torch)."""
    def step(zz):
        return 0.5 * (1.0 + xp.tanh(zz / width))
    dx, dy, dz = x - center[0], y - center[1], z - center[2]
    r = xp.sqrt(dx * dx + dy * dy + dz * dz) + 1e-300
    s_in = step(r - (r_shell - shell))
    s_out = step(r - r_shell)
    rho = rho_in + (rho_shell - rho_in) * s_in + (rho_amb - rho_shell) * s_out
    p = p_in * (1.0 - s_out) + p_amb * s_out
    Ur = U_shell * xp.clamp(r / r_shell, max=1.0) if xp is not np else \
        U_shell * np.minimum(r / r_shell, 1.0)
    Ur = Ur * (1.0 - s_out)
    return xp.stack([rho, Ur * dx / r, Ur * dy / r, Ur * dz / r, p])


def amr_blast_hierarchy(base: int = 64, levels: int = 5, center=(0.6, 0.5, 0.5),
                        r_shell: float = 0.18, widths=(0.06, 0.03, 0.012, 0.004)):
    """Octree of 8^3 patches on [0, 1]^3 (level l has cell size 1/(base 2^l)).
    Level 0 holds all (base/8)^3 patches; a level-l patch is refined into its
    8 children on level l+1 when its box comes within widths[l] of the shell
    |x - center| = r_shell (the region where the gradient criterion fires on
    the blast profile). Returns a list of (n_l, 3) int arrays (ix, iy, iz)."""
    c = np.asarray(center)
    n0 = base // PATCH
    g = np.stack(np.meshgrid(np.arange(n0), np.arange(n0), np.arange(n0), indexing="ij"), -1)
    lev = [g.reshape(-1, 3)[:, ::-1].copy()]  # (ix, iy, iz) with x fastest in the ordering
    lev[0] = lev[0][np.lexsort((lev[0][:, 0], lev[0][:, 1], lev[0][:, 2]))]
    for l in range(levels - 1):
        size = PATCH / (base * 2 ** l)
        lo = lev[l] * size
        hi = lo + size
        near = np.clip(c, lo, hi)
        dmin = np.linalg.norm(near - c, axis=1)
        far = np.where(np.abs(lo - c) > np.abs(hi - c), lo, hi)
        dmax = np.linalg.norm(far - c, axis=1)
        flag = (dmin <= r_shell + widths[l]) & (dmax >= r_shell - widths[l])
        parents = lev[l][flag]
        kids = (parents[:, None, :] * 2 + np.array([[i, j, k] for k in (0, 1) for j in (0, 1)
                                                     for i in (0, 1)])[None]).reshape(-1, 3)
        kids = kids[np.lexsort((kids[:, 0], kids[:, 1], kids[:, 2]))]
        lev.append(kids)
    return lev


def amr_patch_prims(coords, level: int, base: int = 64, xp=np, device=None, **blast):
    """[n][5][12][12][12] primitive values of the blast profile on the ghosted
    patches (ix, iy, iz) of one level; ghost cells take the analytic profile
    at the level's cell size. With xp=torch the values are made on `device`."""
    dh = 1.0 / (base * 2 ** level)
    if xp is np:
        c = np.asarray(coords, dtype=np.float64)
        g = np.arange(GP, dtype=np.float64) - GHOST + 0.5
    else:
        c = xp.as_tensor(np.asarray(coords), dtype=xp.float64, device=device)
        g = xp.arange(GP, dtype=xp.float64, device=device) - GHOST + 0.5
    x = (c[:, 0:1] * PATCH + g[None, :]) * dh    # [n][12]
    y = (c[:, 1:2] * PATCH + g[None, :]) * dh
    z = (c[:, 2:3] * PATCH + g[None, :]) * dh
    X = x[:, None, None, :]
    Y = y[:, None, :, None]
    Z = z[:, :, None, None]
    W = blast_prims_at(X + 0 * Y + 0 * Z, Y + 0 * X + 0 * Z, Z + 0 * X + 0 * Y, xp=xp, **blast)
    return W.transpose(0, 1) if xp is not np else W.transpose(1, 0, 2, 3, 4)


# ---- AMR hierarchies with data exchange (Hierarchy / AmrRun) -----------------

def nested_hierarchy(base=(4, 4, 4), nlev=3):
    """Test hierarchy: level 0 covers the base patches; level l + 1 refines
    the central 2x2x2 patches of level l (a block of 4x4x4 patches at every
    level), so every level's ghost zones lie on its own level or the next
    coarser one. Returns per-level (n_l, 3) patch coordinates."""
    px, py, pz = base
    lev = [np.array([(x, y, z) for z in range(pz) for y in range(py) for x in range(px)])]
    for l in range(1, nlev):
        P = [b << (l - 1) for b in base]
        c = [p // 2 - 1 for p in P]
        lev.append(np.array([(2 * X + cx, 2 * Y + cy, 2 * Z + cz)
                             for Z in (c[2], c[2] + 1) for Y in (c[1], c[1] + 1)
                             for X in (c[0], c[0] + 1)
                             for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]))
    return lev


def level_prims(coords, level, fn, dh0, xp=np, device=None):
    """[n][5][8][8][8] primitive states of level-`level` patches at `coords`,
    fn(x, y, z) -> (rho, Ux, Uy, Uz, p) evaluated at the cell centres
    (physical coordinates, level-0 cell size dh0)."""
    c = xp.asarray(np.asarray(coords), dtype=xp.float64)
    if device is not None:
        c = c.to(device)
    dh = dh0 / 2 ** level
    g = (xp.arange(8, dtype=xp.float64) + 0.5) * dh
    if device is not None:
        g = g.to(device)
    x = 8 * dh * c[:, 0, None, None, None] + g[None, None, None, :]
    y = 8 * dh * c[:, 1, None, None, None] + g[None, None, :, None]
    z = 8 * dh * c[:, 2, None, None, None] + g[None, :, None, None]
    x, y, z = xp.broadcast_arrays(x, y, z) if xp is np else xp.broadcast_tensors(x, y, z)
    W = fn(x, y, z)
    return xp.stack([xp.asarray(w) * xp.ones_like(x) for w in W], 1) if xp is np else \
        xp.stack([w * xp.ones_like(x) for w in W], 1)


def bump_prims(x, y, z, xp=np):
    """Smooth test state for AMR runs: a density and pressure bump moving
    diagonally through the refined block (rho 1..3, p 0.5..1.5, U 0.3)."""
    r2 = (x - 0.45) ** 2 + (y - 0.5) ** 2 + (z - 0.55) ** 2
    e = xp.exp(-r2 / 0.01)
    return (1.0 + 2.0 * e, 0.3 + 0 * x, -0.2 + 0 * x, 0.1 + 0 * x, 0.5 + e)


def jet_hierarchy(base=(8, 8, 16), radii=(0.25, 0.125, 0.0625), heights=(1.0, 0.75, 0.5)):
    """Static hierarchy of the relativistic-jet configuration: level 0 covers
    the base patches ([0,1] x [0,1] x [0,2] in units of the x width); level
    l = 1, 2, 3 refines, in groups of eight, every level-(l-1) patch whose
    box comes within radii[l-1] of the jet axis (x = y = 0.5) and starts
    below heights[l-1] (the cocoon region around the beam), and that is
    surrounded by refined-or-refinable neighbours so that proper nesting
    holds. Returns per-level (n_l, 3) patch coordinates."""
    lev = [np.array([(x, y, z) for z in range(base[2]) for y in range(base[1])
                     for x in range(base[0])])]
    Lx = 1.0
    for l in range(1, len(radii) + 1):
        P = [b << (l - 1) for b in base]
        w = Lx / P[0]  # patch width at level l - 1
        parents = []
        have = set(map(tuple, lev[l - 1]))
        for (X, Y, Z) in lev[l - 1]:
            # distance from the axis to the patch box, and its bottom
            dx = max(abs((X + 0.5) * w - 0.5) - 0.5 * w, 0.0)
            dy = max(abs((Y + 0.5) * w - 0.5) - 0.5 * w, 0.0)
            if np.hypot(dx, dy) <= radii[l - 1] and Z * w < heights[l - 1] * 2 * Lx:
                # proper nesting: all 26 neighbours must exist on level l - 1
                ok = True
                for oz in (-1, 0, 1):
                    for oy in (-1, 0, 1):
                        for ox in (-1, 0, 1):
                            q = (X + ox, Y + oy, Z + oz)
                            inside = all(0 <= q[a] < P[a] for a in range(3))
                            if inside and q not in have:
                                ok = False
                if ok:
                    parents.append((X, Y, Z))
        lev.append(np.array([(2 * X + cx, 2 * Y + cy, 2 * Z + cz) for (X, Y, Z) in parents
                             for cz in (0, 1) for cy in (0, 1) for cx in (0, 1)]).reshape(-1, 3))
    return lev


def jet_states(gamma_jet=10.0, rho_amb=1.0, T_amb=1e-6, density_contrast=1e-3, T_jet=10.0):
    """Primitive states (rho, Ux, Uy, Uz, p) of the cold static ambient and
    of the hot jet beam moving along +z with Lorentz factor gamma_jet."""
    amb = (rho_amb, 0.0, 0.0, 0.0, rho_amb * T_amb)
    rj = rho_amb * density_contrast
    jet = (rj, 0.0, 0.0, float(np.sqrt(gamma_jet ** 2 - 1.0)), rj * T_jet)
    return amb, jet
