"""CPU check of the index maps of the VL patch kernel (srhd_vl.cuh), restated
here: the cells whose state at t^n the predictor reads (N, 1952 cells of
the 14^3 tile), the cells whose half-step state the corrector reads (H,
1280), the predictor faces of each direction (1408) and the inverse maps.
Every map is a bijection onto its set, every index lies in its buffer, and
every value a phase reads was written by an earlier phase."""
import itertools

TILE = 14
N_CELLS, H_CELLS, P_FACES = 1952, 1280, 1408


def t14(i, j, k):
    return ((k + 3) * TILE + (j + 3)) * TILE + (i + 3)


def place(axis, along, u, v):
    return [(along, u, v), (u, along, v), (u, v, along)][axis]


def vl_n_cell(r):
    if r < 512:
        return r & 7, (r >> 3) & 7, r >> 6
    if r < 1664:
        q = r - 512
        f, rem = q // 192, q % 192
        depth, t = 1 + rem // 64, rem % 64
        axis, side = f >> 1, f & 1
        along = 7 + depth if side else -depth
        return place(axis, along, t & 7, t >> 3)
    q = r - 1664
    pair, rem = q // 96, q % 96
    e, rem2 = rem // 24, rem % 24
    dc, w = rem2 // 8, rem2 % 8
    da, db = [(1, 1), (1, 2), (2, 1)][dc]
    ca = 7 + da if e & 1 else -da
    cb = 7 + db if e & 2 else -db
    return [(ca, cb, w), (ca, w, cb), (w, ca, cb)][pair]


def vl_h_cell(r):
    if r < 512:
        return r & 7, (r >> 3) & 7, r >> 6
    q = r - 512
    f6, rem = q >> 7, q & 127
    depth, t = 1 + (rem >> 6), rem & 63
    axis, side = f6 >> 1, f6 & 1
    along = 7 + depth if side else -depth
    return place(axis, along, t & 7, t >> 3)


def h_index(i, j, k):
    c = (i, j, k)
    out = [d for d in range(3) if not 0 <= c[d] <= 7]
    if not out:
        return (k * 8 + j) * 8 + i
    d = out[0]
    x = c[d]
    side = 1 if x > 7 else 0
    depth = x - 7 if side else -x
    u, v = [(j, k), (i, k), (i, j)][d]
    return 512 + (2 * d + side) * 128 + (depth - 1) * 64 + v * 8 + u


def pface(r):
    """r -> (f, a, b): face between cells f-1 and f along d, transverse (a, b)."""
    if r < 832:
        return -2 + r % 13, (r // 13) & 7, (r // 13) >> 3
    q = r - 832
    g, rem = q // 288, q % 288
    f, t = rem % 9, rem // 9
    o = (-2, -1, 8, 9)[t & 3]
    w = t >> 2
    return (f, o, w) if g == 0 else (f, w, o)


def pface_index(f, a, b):
    if 0 <= a <= 7 and 0 <= b <= 7:
        return (b * 8 + a) * 13 + (f + 2)
    g = 0 if not 0 <= a <= 7 else 1
    o, w = (a, b) if g == 0 else (b, a)
    io = o + 2 if o < 0 else o - 6
    return 832 + g * 288 + (w * 4 + io) * 9 + f


def cell_of(d, x, a, b):
    return [(x, a, b), (a, x, b), (a, b, x)][d]


def depth(x):
    return -x if x < 0 else (x - 7 if x > 7 else 0)


def test_sets_are_the_stencil_closures():
    n_set = [vl_n_cell(r) for r in range(N_CELLS)]
    h_set = [vl_h_cell(r) for r in range(H_CELLS)]
    assert len(set(n_set)) == N_CELLS and len(set(h_set)) == H_CELLS
    # H: the cells whose half-step state the corrector's slopes read
    need_h = set()
    for d in range(3):
        for f in range(9):
            for a, b in itertools.product(range(8), range(8)):
                for x in (f - 2, f - 1, f, f + 1):
                    need_h.add(cell_of(d, x, a, b))
    assert need_h == set(h_set)
    # predictor faces: both faces along every direction of every H cell
    faces = [set() for _ in range(3)]
    for (i, j, k) in h_set:
        c = (i, j, k)
        for d in range(3):
            a, b = [(j, k), (i, k), (i, j)][d]
            faces[d].add((c[d], a, b))
            faces[d].add((c[d] + 1, a, b))
    for d in range(3):
        listed = [pface(r) for r in range(P_FACES)]
        assert len(set(listed)) == P_FACES and set(listed) == faces[d]
        for r in range(P_FACES):
            assert pface_index(*pface(r)) == r
    # N: the two cells of every predictor face, and the H cells themselves
    need_n = set(h_set)
    for d in range(3):
        for (f, a, b) in faces[d]:
            need_n.add(cell_of(d, f - 1, a, b))
            need_n.add(cell_of(d, f, a, b))
    assert need_n == set(n_set)


def test_indices_in_bounds_and_inverse():
    for r in range(N_CELLS):
        i, j, k = vl_n_cell(r)
        assert all(-3 <= c <= 10 for c in (i, j, k))
        assert 0 <= t14(i, j, k) < TILE ** 3
    for r in range(H_CELLS):
        c = vl_h_cell(r)
        assert h_index(*c) == r
        assert max(depth(x) for x in c) <= 2
    # the corrector's cells along d for faces 0..8 are H cells
    for d in range(3):
        for f in range(9):
            for a, b in itertools.product(range(8), range(8)):
                for x in (f - 2, f - 1, f, f + 1):
                    assert 0 <= h_index(*cell_of(d, x, a, b)) < H_CELLS
