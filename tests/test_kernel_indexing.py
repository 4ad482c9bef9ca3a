"""CPU check of the fused patch kernel's addressing for every launch
variant declared in srhd_launch.inl: every shared-memory, face-slot, tile
and output index that the work loops produce (for each thread of a CTA of
that size, with and without the paired Newton solves) lies inside its
buffer. The loop bounds and index maps restate those of srhd_kernels.cuh;
a variant whose loops would leave a buffer is caught here, on the CPU,
before it runs on a GPU."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
kG, kGC, kNC, kNF, kRC, NEED = 12, 1728, 512, 576, 896, 1376


def _variants():
    src = open(os.path.join(ROOT, "paper_2012_11130_gb300", "csrc", "srhd_launch.inl")).read()
    pat = (r"struct PatchVariant<(double|float), (\d)> \{ static constexpr int nt = (\d+), "
           r"minb = (\d+); static constexpr bool pair = (true|false); \}")
    out = [(t, int(v), int(nt), int(mb), p == "true") for t, v, nt, mb, p in re.findall(pat, src)]
    assert len(out) == 8
    return out


def needed_tile_cell(r):
    if r < 512:
        g = [2 + (r & 7), 2 + ((r >> 3) & 7), 2 + (r >> 6)]
    elif r < 1280:
        q = r - 512
        f, rem = q >> 7, q & 127
        axis, depth, t = f >> 1, 1 + (rem >> 6), rem & 63
        along = 9 + depth if (f & 1) else 2 - depth
        u, v = 2 + (t & 7), 2 + (t >> 3)
        g = [along, u, v] if axis == 0 else ([u, along, v] if axis == 1 else [u, v, along])
    else:
        q = r - 1280
        e, w = q >> 3, 2 + (q & 7)
        ca, cb = (10 if e & 1 else 1), (10 if e & 2 else 1)
        g = [[ca, cb, w], [ca, w, cb], [w, ca, cb]][e >> 2]
    return (g[2] * 12 + g[1]) * 12 + g[0]


def recon_cell(r):
    if r < kNC:
        return r & 7, (r >> 3) & 7, r >> 6
    r -= kNC
    layer, q = r >> 6, r & 63
    a, b = q & 7, q >> 3
    side = 8 if (layer & 1) else -1
    return [(side, a, b), (a, side, b), (a, b, side)][layer >> 1]


def tile_index(i, j, k):
    return ((k + 2) * kG + (j + 2)) * kG + (i + 2)


def face_index(d, i, j, k, fd):
    return [(k * 8 + j) * 9 + fd, (k * 9 + fd) * 8 + i, (fd * 8 + j) * 8 + i][d]


def face_owner(d, fi, side):
    if d == 0:
        fd, j, k = fi % 9, (fi // 9) & 7, fi // 72
        i = fd - 1 + side
    elif d == 1:
        i, fd, k = fi & 7, (fi >> 3) % 9, (fi >> 3) // 9
        j = fd - 1 + side
    else:
        i, j, fd = fi & 7, (fi >> 3) & 7, fi >> 6
        k = fd - 1 + side
    return tile_index(i, j, k)


def test_tile_cell_list_is_the_read_set():
    def gclass(g):
        return 0 if 2 <= g <= 9 else (1 if g in (1, 10) else 2)

    def needed(c):
        a, b, cc = gclass(c % 12), gclass((c // 12) % 12), gclass(c // 144)
        n = (a > 0) + (b > 0) + (cc > 0)
        return n <= 1 or (n == 2 and max(a, b, cc) <= 1)
    cells = [needed_tile_cell(r) for r in range(NEED)]
    assert len(set(cells)) == NEED and set(cells) == {c for c in range(kGC) if needed(c)}


@pytest.mark.parametrize("var", _variants(), ids=lambda v: f"{v[0]}-{v[1]}")
def test_variant_indices_in_bounds(var):
    _, _, NT, _, PAIR = var
    assert NT % 32 == 0
    bad = []

    def chk(name, val, hi):
        if not (0 <= val < hi):
            bad.append((name, val))
    for tid in range(NT):
        if PAIR:
            for r in range(tid, NEED // 2, NT):
                chk("tile", needed_tile_cell(r), kGC)
                chk("tile", needed_tile_cell(r + NEED // 2), kGC)
        else:
            for r in range(tid, NEED, NT):
                chk("tile", needed_tile_cell(r), kGC)
        for r in range(tid, kRC, NT):
            i, j, k = recon_cell(r)
            tc = tile_index(i, j, k)
            for d, off in ((0, 1), (1, 12), (2, 144)):
                chk("nb", tc - off, kGC)
                chk("nb", tc + off, kGC)
                cd = (i, j, k)[d]
                trans = r < kNC or cd < 0 or cd > 7
                if trans and cd >= 0:
                    chk("slot", face_index(d, i, j, k, cd), kNF)
                if trans and cd <= 7:
                    chk("slot", face_index(d, i, j, k, cd + 1), kNF)
        for f in range(tid, 3 * kNF, NT):
            d, fi = f // kNF, f % kNF
            chk("owner", face_owner(d, fi, 0), kGC)
            chk("owner", face_owner(d, fi, 1), kGC)
        npc = 2 if PAIR else 1
        items = kNC // npc
        for c0 in range(tid, items, NT):
            for q in range(npc):
                c = c0 + q * items
                chk("cell", c, kNC)
                i, j, k = c & 7, (c >> 3) & 7, c >> 6
                chk("tc", tile_index(i, j, k), kGC)
                for d, cd in ((0, i), (1, j), (2, k)):
                    chk("face", face_index(d, i, j, k, cd + 1), kNF)
                chk("out", 4 * kNC + c, 5 * kNC)
        chk("red", tid >> 5, NT // 32)
    assert not bad, bad[:5]


def face_slot(d, side, v):
    """Offset of face slot (d, side, v): side-major, [side][d][v][576]."""
    return ((side * 3 + d) * 5 + v) * kNF


@pytest.mark.parametrize("elem", [4, 8])
def test_stage_region_is_the_right_state_slots(elem):
    # The next patch's ghosted tile (5 x 12^3 elements) is copied into the
    # right-state slots (side 1) during phase 4; phase 4 and the outputs read
    # only the flux slots (side 0), which must not overlap it.
    stage0, stage_len = 3 * 5 * kNF, 5 * kGC
    assert stage_len == 3 * 5 * kNF
    offs = sorted(face_slot(d, s, v) for d in range(3) for s in range(2) for v in range(5))
    assert offs == [q * kNF for q in range(30)]          # 30 disjoint slots fill the region
    side1 = {face_slot(d, 1, v) + i for d in range(3) for v in range(5) for i in (0, kNF - 1)}
    assert min(side1) == stage0 and max(side1) == stage0 + stage_len - 1
    for d in range(3):
        for v in range(5):
            assert face_slot(d, 0, v) + kNF <= stage0      # flux slots end before the stage
    # copy sizes and addresses: one copy per variable of kGC elements, tiles
    # of 5 kGC elements; shared offset of the stage after the primitive tile
    assert (kGC * elem) % 16 == 0 and (5 * kGC * elem) % 16 == 0
    assert ((5 * kGC + stage0) * elem) % 16 == 0
