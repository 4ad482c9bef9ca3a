"""CPU check of the index arithmetic of the uniform ghost-fill kernel
(fill_ghosts_kernel in srhd_kernels.cuh), restated here: every source index
lies in the interior array, every destination in the ghosted rows of the
range, the rows tile each ghosted patch exactly once, the vector stores are
aligned, and the gathered values equal a wrap/edge padding of the field."""
import numpy as np
import pytest

KN = 8


def ghost_src(g, pc, n, bc):
    o = -1 if g < 0 else (1 if g >= KN else 0)
    q, l = pc + o, g - KN * o
    if q < 0 or q >= n:
        if bc == 0:
            q = q + n if q < 0 else q - n
        else:
            q, l = pc, (0 if o < 0 else KN - 1)
    return q, l


def kernel_fill(interior, npx, npy, npz, bc, gh, p0, nfill):
    """The kernel's loops with its index arithmetic; returns the ghosted rows
    and checks every index against its array."""
    te = KN + 2 * gh
    tc, rows = te ** 3, 5 * te * te
    flat = interior.reshape(-1)
    out = np.full(nfill * 5 * tc, np.nan)
    written = np.zeros(out.size, int)
    for pl in range(nfill):
        p = p0 + pl
        px, py, pz = p % npx, (p // npx) % npy, p // (npx * npy)
        qxl, qxr, cl, cr = px - 1, px + 1, False, False
        if qxl < 0:
            if bc[0] == 0:
                qxl += npx
            else:
                qxl, cl = px, True
        if qxr >= npx:
            if bc[0] == 0:
                qxr -= npx
            else:
                qxr, cr = px, True
        for r in range(rows):
            v, rem = r // (te * te), r % (te * te)
            tz, ty = rem // te, rem % te
            qz, lz = ghost_src(tz - gh, pz, npz, bc[2])
            qy, ly = ghost_src(ty - gh, py, npy, bc[1])
            plane = (qz * npy + qy) * npx
            cell = (lz * KN + ly) * KN
            src = []
            for i in range(gh):
                src.append(((plane + qxl) * 5 + v) * 512 + cell + (0 if cl else KN - gh + i))
            for i in range(KN):
                src.append(((plane + px) * 5 + v) * 512 + cell + i)
            for i in range(gh):
                src.append(((plane + qxr) * 5 + v) * 512 + cell + (KN - 1 if cr else i))
            dst = pl * 5 * tc + r * te
            assert all(0 <= s < flat.size for s in src)
            assert 0 <= dst and dst + te <= out.size
            out[dst:dst + te] = flat[src]
            written[dst:dst + te] += 1
    assert (written == 1).all()
    return out.reshape(nfill, 5, te, te, te)


@pytest.mark.parametrize("gh", [2, 3])
@pytest.mark.parametrize("dims,bc", [((3, 2, 4), (0, 0, 0)), ((3, 2, 4), (1, 0, 1)),
                                     ((1, 1, 2), (0, 1, 0)), ((2, 1, 1), (1, 1, 1))])
def test_fill_matches_padding(gh, dims, bc):
    npx, npy, npz = dims
    rng = np.random.default_rng(7)
    field = rng.normal(size=(5, 8 * npz, 8 * npy, 8 * npx))
    patches = field.reshape(5, npz, 8, npy, 8, npx, 8).transpose(1, 3, 5, 0, 2, 4, 6)
    patches = patches.reshape(-1, 5, 8, 8, 8)
    padded = field
    for ax, b in zip((3, 2, 1), bc):
        pads = [(0, 0)] * 4
        pads[ax] = (gh, gh)
        padded = np.pad(padded, pads, mode="wrap" if b == 0 else "edge")
    te = KN + 2 * gh
    n = npx * npy * npz
    for p0, nf in ((0, n), (n // 2, n - n // 2)):
        G = kernel_fill(patches, npx, npy, npz, bc, gh, p0, nf)
        for pl in range(nf):
            p = p0 + pl
            px, py, pz = p % npx, (p // npx) % npy, p // (npx * npy)
            want = padded[:, 8 * pz:8 * pz + te, 8 * py:8 * py + te, 8 * px:8 * px + te]
            assert np.array_equal(G[pl], want)


@pytest.mark.parametrize("esz", [4, 8])
@pytest.mark.parametrize("gh", [2, 3])
def test_vector_stores_aligned(esz, gh):
    te = KN + 2 * gh
    align = 8 if (esz == 4 and te % 4 != 0) else 16
    width = 4 if (esz == 4 and te % 4 == 0) else 2     # elements per store
    assert te % width == 0 and width * esz == align
    tile = 5 * te ** 3 * esz
    assert tile % align == 0 and (te * esz) % align == 0


def tile_src(c, gp, dims, bc, nvar=5):
    """The patch kernel's gather offset of 12^3 tile cell c of grid patch gp
    in an array [np][nvar][8^3] (nvar 5: the conserved interiors; 6: the
    primitive cache of srhd_advance_uniform_prim)."""
    npx, npy, npz = dims
    gpx, gpy, gpz = gp % npx, (gp // npx) % npy, gp // (npx * npy)
    gz, gy, gx = c // 144, (c // 12) % 12, c % 12
    qx, lx = ghost_src(gx - 2, gpx, npx, bc[0])
    qy, ly = ghost_src(gy - 2, gpy, npy, bc[1])
    qz, lz = ghost_src(gz - 2, gpz, npz, bc[2])
    return ((qz * npy + qy) * npx + qx) * (nvar * 512) + (lz * 8 + ly) * 8 + lx


@pytest.mark.parametrize("nvar", [5, 6])
@pytest.mark.parametrize("dims,bc", [((3, 2, 4), (0, 0, 0)), ((3, 2, 4), (1, 0, 1)),
                                     ((1, 1, 1), (0, 1, 0))])
def test_gather_offsets_match_padding(dims, bc, nvar):
    npx, npy, npz = dims
    rng = np.random.default_rng(3)
    field = rng.normal(size=(nvar, 8 * npz, 8 * npy, 8 * npx))
    flat = field.reshape(nvar, npz, 8, npy, 8, npx, 8).transpose(1, 3, 5, 0, 2, 4, 6).reshape(-1)
    padded = field
    for ax, b in zip((3, 2, 1), bc):
        pads = [(0, 0)] * 4
        pads[ax] = (2, 2)
        padded = np.pad(padded, pads, mode="wrap" if b == 0 else "edge")
    for gp in range(npx * npy * npz):
        px, py, pz = gp % npx, (gp // npx) % npy, gp // (npx * npy)
        want = padded[:, 8 * pz:8 * pz + 12, 8 * py:8 * py + 12, 8 * px:8 * px + 12]
        off = np.array([tile_src(c, gp, dims, bc, nvar) for c in range(1728)])
        assert off.min() >= 0 and off.max() + (nvar - 1) * 512 < flat.size
        for v in range(nvar):
            assert np.array_equal(flat[off + v * 512], want[v].reshape(-1))
        # the interior cells' own offsets (phase 4) are gp*nvar*512 + c
        for c in (0, 7, 63, 511):
            i, j, k = c & 7, (c >> 3) & 7, c >> 6
            assert (tile_src(((k + 2) * 12 + j + 2) * 12 + i + 2, gp, dims, bc, nvar)
                    == gp * nvar * 512 + c)


# Staged uniform gather (tensor maps): box layout of the stage and the
# offsets box_offset gives, restated from srhd_kernels.cuh.
KBOX_C, KBOX_X, KBOX_Y, KBOX_Z = 2560, 1280, 640, 640
KXM = KBOX_C
KXP, KYM = KXM + KBOX_X, KXM + 2 * KBOX_X
KYP, KZM = KYM + KBOX_Y, KYM + 2 * KBOX_Y
KZP = KZM + KBOX_Z


def box_offset(gx, gy, gz):
    ax = 0 if gx < 2 else (1 if gx < 10 else 2)
    ay = 0 if gy < 2 else (1 if gy < 10 else 2)
    az = 0 if gz < 2 else (1 if gz < 10 else 2)
    x, y, z = gx - 2, gy - 2, gz - 2
    if ay == 1 and az == 1:
        if ax == 1:
            return (z * 8 + y) * 8 + x, 512
        return (KXM + gx + 2 if ax == 0 else KXP + gx - 10) + (z * 8 + y) * 4, 256
    if ax == 1 and az == 1:
        return (KYM + gy * 8 if ay == 0 else KYP + (gy - 10) * 8) + z * 16 + x, 128
    if ax == 1 and ay == 1:
        return (KZM + gz * 64 if az == 0 else KZP + (gz - 10) * 64) + y * 8 + x, 128
    return None


def test_staged_boxes_give_the_tile():
    # boxes as the tensor copies deliver them (dense, x fastest) for a patch
    # of a periodic grid, against numpy.pad of the whole field
    from test_kernel_indexing import NEED, needed_tile_cell
    npx, npy, npz = 3, 4, 5
    rng = np.random.default_rng(8)
    field = rng.normal(size=(5, 8 * npz, 8 * npy, 8 * npx))
    P = field.reshape(5, npz, 8, npy, 8, npx, 8).transpose(1, 3, 5, 0, 2, 4, 6)  # [z][y][x][v][8][8][8]
    padded = np.pad(field, [(0, 0), (2, 2), (2, 2), (2, 2)], mode="wrap")
    needed = [needed_tile_cell(r) for r in range(NEED)]
    for (cz, cy, cx) in ((0, 0, 0), (2, 1, 1), (4, 3, 2)):
        nb = lambda dz, dy, dx: P[(cz + dz) % npz, (cy + dy) % npy, (cx + dx) % npx]  # noqa: E731
        stage = np.full(KZP + KBOX_Z, np.nan)
        stage[0:KBOX_C] = nb(0, 0, 0).reshape(-1)                       # [v][z][y][x]
        stage[KXM:KXM + KBOX_X] = nb(0, 0, -1)[:, :, :, 4:8].reshape(-1)
        stage[KXP:KXP + KBOX_X] = nb(0, 0, 1)[:, :, :, 0:4].reshape(-1)
        stage[KYM:KYM + KBOX_Y] = nb(0, -1, 0)[:, :, 6:8, :].reshape(-1)
        stage[KYP:KYP + KBOX_Y] = nb(0, 1, 0)[:, :, 0:2, :].reshape(-1)
        stage[KZM:KZM + KBOX_Z] = nb(-1, 0, 0)[:, 6:8, :, :].reshape(-1)
        stage[KZP:KZP + KBOX_Z] = nb(1, 0, 0)[:, 0:2, :, :].reshape(-1)
        want = padded[:, 8 * cz:8 * cz + 12, 8 * cy:8 * cy + 12, 8 * cx:8 * cx + 12]
        nstaged = 0
        for c in needed:
            gz, gy, gx = c // 144, (c // 12) % 12, c % 12
            got = box_offset(gx, gy, gz)
            nout = sum(1 for g in (gx, gy, gz) if g < 2 or g > 9)
            if got is None:
                assert nout == 2            # only the first-layer edges are not staged
                continue
            off, vs = got
            assert 0 <= off and off + 4 * vs < KZP + KBOX_Z
            for v in range(5):
                assert stage[off + v * vs] == want[v, gz, gy, gx]
            nstaged += 1
        assert nstaged == NEED - 96
    # every box starts on a 128-byte boundary for 4- and 8-byte elements
    for off in (0, KXM, KXP, KYM, KYP, KZM, KZP):
        assert (off * 4) % 128 == 0


@pytest.mark.parametrize("elem", [4, 8])
def test_tensor_copy_coordinates(elem):
    # The seven boxes of the staged uniform gather (box dims x, y, z and
    # start coordinates, restated from the issue code in srhd_kernels.cuh;
    # all seven are tensor copies in mode 3, the x and y slabs in mode 1,
    # whose centre and z slabs test_bulk_copies_of_the_uniform_stage covers):
    # the innermost start x times the element size must be a multiple of 16
    # bytes, every box must lie inside the patch, and the bytes the mbarrier
    # expects must be the sum of the boxes.
    boxes = {"center": ((8, 8, 8), (0, 0, 0)), "-x": ((4, 8, 8), (4, 0, 0)),
             "+x": ((4, 8, 8), (0, 0, 0)), "-y": ((8, 2, 8), (0, 6, 0)),
             "+y": ((8, 2, 8), (0, 0, 0)), "-z": ((8, 8, 2), (0, 0, 6)),
             "+z": ((8, 8, 2), (0, 0, 0))}
    total = 0
    for (bx, by, bz), (x0, y0, z0) in boxes.values():
        assert (x0 * elem) % 16 == 0 and (bx * elem) % 16 == 0
        assert 0 <= x0 and x0 + bx <= 8 and 0 <= y0 and y0 + by <= 8 and 0 <= z0 and z0 + bz <= 8
        total += bx * by * bz * 5
    assert total == KZP + KBOX_Z == 7680
    # the neighbour slabs hold the cells the tile needs: x 6, 7 of the -x
    # neighbour inside [4, 8), y 6, 7 of the -y neighbour, and so on
    assert {6, 7} <= set(range(4, 8)) and {0, 1} <= set(range(0, 4))


def staged_cell(r):
    """Restatement of staged_cell (srhd_kernels.cuh): tile index, stage
    offset, variable stride, holding patch (0 itself, 1 + face) and the
    cell's 8^3 index there, for the needed cells r < 1280."""
    def tile_index(i, j, k):
        return ((k + 2) * 12 + j + 2) * 12 + i + 2
    if r < 512:
        return tile_index(r & 7, (r >> 3) & 7, r >> 6), r, 512, 0, r
    q = r - 512
    f, rem = q >> 7, q & 127
    depth, t = 1 + (rem >> 6), rem & 63
    a, b = t & 7, t >> 3
    lo, hi = 8 - depth, depth - 1
    if f == 0:
        return tile_index(-depth, a, b), KXM + 4 - depth + 4 * t, 256, 1, t * 8 + lo
    if f == 1:
        return tile_index(7 + depth, a, b), KXP + hi + 4 * t, 256, 2, t * 8 + hi
    if f == 2:
        return tile_index(a, -depth, b), KYM + (2 - depth) * 8 + b * 16 + a, 128, 3, (b * 8 + lo) * 8 + a
    if f == 3:
        return tile_index(a, 7 + depth, b), KYP + hi * 8 + b * 16 + a, 128, 4, (b * 8 + hi) * 8 + a
    if f == 4:
        return tile_index(a, b, -depth), KZM + (2 - depth) * 64 + t, 128, 5, lo * 64 + t
    return tile_index(a, b, 7 + depth), KZP + hi * 64 + t, 128, 6, hi * 64 + t


def test_closed_form_staged_cells_match_box_offset_and_sources():
    # The closed-form mapping of the staged gather (modes 1 and 3) gives, for
    # every interior and face-slab cell of the needed list, the tile cell of
    # needed_tile_cell, the stage offset and stride of box_offset, and the
    # patch and cell that ghost_src finds (periodic grid, interior patch).
    from test_kernel_indexing import needed_tile_cell
    faces = {0: (0, 0, 0), 1: (-1, 0, 0), 2: (1, 0, 0), 3: (0, -1, 0), 4: (0, 1, 0),
             5: (0, 0, -1), 6: (0, 0, 1)}
    for r in range(512 + 768):
        c, off, vs, nb, local = staged_cell(r)
        assert c == needed_tile_cell(r)
        gz, gy, gx = c // 144, (c // 12) % 12, c % 12
        assert box_offset(gx, gy, gz) == (off, vs)
        # the source by plain geometry: patch offset and cell of (g - 2)
        src = []
        for g in (gx, gy, gz):
            o = -1 if g - 2 < 0 else (1 if g - 2 >= 8 else 0)
            src.append((o, g - 2 - 8 * o))
        assert tuple(s[0] for s in src) == faces[nb]
        assert (src[2][1] * 8 + src[1][1]) * 8 + src[0][1] == local


def test_bulk_copies_of_the_uniform_stage():
    # Mode 1 stages the patch interior and the two z slabs with plain bulk
    # copies (the x and y slabs stay tensor boxes): the interior is one run of
    # 5 x 512 values; each z slab is, per variable, the 128 values of two
    # planes (z 6, 7 of the -z neighbour at offset 384; z 0, 1 of the +z
    # one at 0), landing at stage offsets KZM/KZP + 128 v: the layout of the
    # [5][2][8][8] boxes. Every copy starts and ends on 16 bytes.
    field = np.arange(5 * 512, dtype=np.float64).reshape(5, 8, 8, 8)  # [v][z][y][x]
    zm = field[:, 6:8].reshape(5, 128)
    zp = field[:, 0:2].reshape(5, 128)
    flat = field.reshape(-1)
    for v in range(5):
        assert np.array_equal(flat[v * 512 + 384:v * 512 + 512], zm[v])
        assert np.array_equal(flat[v * 512:v * 512 + 128], zp[v])
    for elem in (4, 8):
        for off, n in [(0, 2560)] + [(v * 512 + 384, 128) for v in range(5)]:
            assert (off * elem) % 16 == 0 and (n * elem) % 16 == 0
        for st in (0, KZM, KZP):
            assert (st * elem) % 16 == 0
    assert KZP + KBOX_Z - KZM == 2 * 5 * 128
