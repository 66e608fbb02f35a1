"""Pins for the CPU oracle: closed forms, hand-derived counts, an independent exact method and
invariants, so that a plausible mistake in the oracle (a dropped closing edge, a wrong tie
direction, a transposed x/y, an off-by-one pixel window, a wrong union) fails at least one test.

Nothing here comes from the CUDA path."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W


def rect(x0, y0, w, h):
    return [[x0, y0], [x0 + w, y0], [x0 + w, y0 + h], [x0, y0 + h]]


# ------------------------------------------------------------------------------- closed forms

def test_unit_square():
    assert O.polygon_area(rect(0, 0, 1, 1)) == 1
    assert O.polygon_area(rect(-7, 12, 1, 1)) == 1


@pytest.mark.parametrize("method", ["brute", "rle"])
def test_rectangles_area_is_w_times_h(method):
    rng = np.random.default_rng(11)
    area = O.polygon_area if method == "brute" else O.polygon_area_rle
    for _ in range(200):
        x0, y0 = (int(v) for v in rng.integers(-1000, 1000, 2))
        w, h = (int(v) for v in rng.integers(1, 40, 2))
        r = rect(x0, y0, w, h)
        assert area(r) == w * h
        assert area(r[::-1]) == w * h          # clockwise ring: same pixels
        assert area(r[2:] + r[:2]) == w * h    # ring rotated: same polygon


@pytest.mark.parametrize("method", ["brute", "rle"])
def test_rectangle_pairs_exact_overlap(method):
    """||p n q|| of two axis-aligned rectangles is the product of the interval overlaps and
    ||p u q|| = w_p h_p + w_q h_q - ||p n q|| (Sec. 2.2)."""
    rng = np.random.default_rng(12)
    fn = O.pair if method == "brute" else O.pair_rle
    for _ in range(300):
        ax, ay = (int(v) for v in rng.integers(-50, 50, 2))
        aw, ah = (int(v) for v in rng.integers(1, 30, 2))
        bx, by = ax + int(rng.integers(-35, 35)), ay + int(rng.integers(-35, 35))
        bw, bh = (int(v) for v in rng.integers(1, 30, 2))
        ox = max(0, min(ax + aw, bx + bw) - max(ax, bx))
        oy = max(0, min(ay + ah, by + bh) - max(ay, by))
        inter, uni = fn(rect(ax, ay, aw, ah), rect(bx, by, bw, bh))
        assert inter == ox * oy
        assert uni == aw * ah + bw * bh - ox * oy


def test_non_square_rectangle_orientation():
    """A 7 x 2 rectangle has 7 pixels per row and 2 rows: catches a transposed window."""
    r = rect(3, -4, 7, 2)
    assert O.polygon_area(r) == 14
    assert O.pixel_in_polygon(r, 9, -3) == 1      # last column, last row
    assert O.pixel_in_polygon(r, 10, -3) == 0     # one past the right side
    assert O.pixel_in_polygon(r, 9, -2) == 0      # one past the top
    assert O.pixel_in_polygon(r, 3, -4) == 1
    assert O.pixel_in_polygon(r, 2, -4) == 0


# ------------------------------------------------------------------------------- tie rule
#
# Pixel centres that lie exactly on an edge: the edge is not counted (the crossing must be strictly
# to the right of the centre). Expected counts derived by hand, pixel by pixel.

def test_tie_rule_right_triangle_hypotenuse_left_of_ray():
    # (0,0),(4,0),(0,4): hypotenuse x + y = 4. Centres (i+.5, j+.5) with i + j = 3 lie on it; the
    # only edge to their right would be the hypotenuse itself (not counted) -> outside.
    # Inside: i + j <= 2 -> 1 + 2 + 3 = 6 pixels.
    tri = [[0, 0], [4, 0], [0, 4]]
    assert O.polygon_area(tri) == 6
    assert O.pixel_in_polygon(tri, 1, 2) == 0   # on the hypotenuse
    assert O.pixel_in_polygon(tri, 1, 1) == 1


def test_tie_rule_diagonal_with_edge_to_the_right():
    # (0,0),(4,0),(4,4): diagonal y = x. Centres with i = j lie on it; their ray still crosses the
    # vertical side x = 4 -> one crossing -> inside. Inside: j < i (6) plus the diagonal (4) = 10.
    tri = [[0, 0], [4, 0], [4, 4]]
    assert O.polygon_area(tri) == 10
    assert O.pixel_in_polygon(tri, 2, 2) == 1


def test_tie_rule_shared_diagonal_partitions_square():
    # The two triangles sharing the diagonal (0,0)-(4,4) split the 4x4 square: every pixel belongs
    # to exactly one of them (10 + 6 = 16), a property of the strict crossing rule.
    t1 = [[0, 0], [4, 0], [4, 4]]
    t2 = [[0, 0], [4, 4], [0, 4]]
    assert O.polygon_area(t2) == 6
    inter, uni = O.pair(t1, t2)
    assert inter == 0 and uni == 16


def test_tie_rule_diamond():
    # |x-2| + |y-2| <= 2. Strictly inside: the 4 centre pixels. Eight centres lie on edges; the
    # left-hand ones ((0,1), (0,2), (1,0), (1,3)) still see an edge to their right -> inside, the
    # right-hand ones ((3,1), (3,2), (2,0), (2,3)) do not -> outside. Total 8 (= the true area).
    d = [[2, 0], [4, 2], [2, 4], [0, 2]]
    assert O.polygon_area(d) == 8
    got = {(x, y) for x in range(4) for y in range(4) if O.pixel_in_polygon(d, x, y)}
    assert got == {(1, 1), (1, 2), (2, 1), (2, 2), (0, 1), (0, 2), (1, 0), (1, 3)}
    assert O.polygon_area_rle(d) == 8


def test_closing_edge_matters():
    # The implicit closing edge v_{n-1} -> v_0 bounds the polygon on the left; dropping it would
    # make every pixel left of the right side see 1 crossing and the area would change.
    tri = [[0, 0], [6, 0], [6, 3]]
    # slope 1/2 diagonal from (0,0) to (6,3): row j has centres right of x = 2(j + .5): j=0: x>1 ->
    # columns 1..5 (5), j=1: x>3 -> 3..5 (3), j=2: x>5 -> 5 (1) => 9 pixels
    assert O.polygon_area(tri) == 9
    assert O.polygon_area_rle(tri) == 9


# ------------------------------------------------------------------------------- shoelace

@pytest.mark.parametrize("method", ["brute", "rle"])
def test_rectilinear_pixel_count_equals_shoelace_and_column_sum(method):
    """For pixel-aligned rectilinear simple polygons (Fig. 3) the pixel count equals the shoelace
    area (Sec. 3.2, POLYAREA) and the sum of column heights of the construction."""
    rng = np.random.Generator(np.random.PCG64(0))
    rings, heights = W.staircase_rings(rng, 150)
    area = O.polygon_area if method == "brute" else O.polygon_area_rle
    for ring, hh in zip(rings, heights):
        a = area(ring)
        assert a == int(hh.sum())
        assert abs(O.shoelace_area2(ring)) == 2 * a
        assert area(ring[::-1]) == a


# ------------------------------------------------------------------------------- invariants

def test_brute_force_equals_row_intervals_on_single_tile(cfg1):
    w = cfg1
    area_a, mbr_a = O.polygon_areas(w.A.off, w.A.xy, "brute")
    area_a2, mbr_a2 = O.polygon_areas(w.A.off, w.A.xy, "rle")
    np.testing.assert_array_equal(area_a, area_a2)
    np.testing.assert_array_equal(mbr_a, mbr_a2)
    area_b, mbr_b = O.polygon_areas(w.B.off, w.B.xy, "brute")
    pa, pb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    assert 1000 < pa.shape[0] < 3000
    i1, u1 = O.pair_areas(w.A, w.B, pa, pb, "brute")
    i2, u2 = O.pair_areas(w.A, w.B, pa, pb, "rle")
    np.testing.assert_array_equal(i1, i2)
    np.testing.assert_array_equal(u1, u2)
    # union counted directly equals ||p|| + ||q|| - ||p n q|| on every pair
    np.testing.assert_array_equal(u1, area_a[pa] + area_b[pb] - i1)
    assert (i1 > 0).sum() > 700


def test_self_pair_symmetry_and_translation(cfg1):
    w = cfg1
    rng = np.random.default_rng(5)
    for i in rng.choice(w.A.n, 60, replace=False):
        p = w.A.polygon(int(i))
        a = O.polygon_area(p)
        assert O.pair(p, p) == (a, a)
        j = int(rng.integers(0, w.B.n))
        q = w.B.polygon(j)
        assert O.pair(p, q) == O.pair(q, p)
        d = np.array([int(rng.integers(-3000, 3000)), int(rng.integers(-3000, 3000))])
        assert O.pair(p + d, q + d) == O.pair(p, q)
        assert O.polygon_area(p + d) == a


def test_disjoint_windows_give_zero_intersection():
    p = [[0, 0], [10, 3], [4, 9]]
    q = [[20, 20], [30, 22], [25, 31]]
    inter, uni = O.pair(p, q)
    assert inter == 0
    assert uni == O.polygon_area(p) + O.polygon_area(q)


# ------------------------------------------------------------------------------- candidate pairs

def test_candidate_pairs_constructed_grid():
    """A: 10x10 squares on a 20 px lattice. B: the same squares shifted by d in x. Closed MBRs
    touch at |d| = 10, so B(i, j) pairs with A(i, j) always and with A(i+1, j) exactly when d = 10
    and with A(i-1, j) exactly when d = -10. Columns i < 3 lie in tile 0, the rest in tile 1,
    so pairs that would straddle the tile line are excluded."""
    for d in (-10, -9, 0, 7, 10):
        a_rings, a_tiles, a_key = [], [], {}
        for i in range(6):
            for j in range(4):
                a_key[(i, j)] = len(a_rings)
                a_rings.append(rect(20 * i, 20 * j, 10, 10))
                a_tiles.append(0 if i < 3 else 1)
        b_rings, b_tiles, b_key = [], [], {}
        for i in range(6):
            for j in range(4):
                b_key[(i, j)] = len(b_rings)
                b_rings.append(rect(20 * i + d, 20 * j, 10, 10))
                b_tiles.append(0 if i < 3 else 1)
        A = W.from_rings(a_rings, a_tiles)
        B = W.from_rings(b_rings, b_tiles)
        _, ma = O.polygon_areas(A.off, A.xy)
        _, mb = O.polygon_areas(B.off, B.xy)
        pa, pb = O.candidate_pairs(ma, A.tile, mb, B.tile)
        expect = set()
        for (i, j), bi in b_key.items():
            expect.add((a_key[(i, j)], bi))
            if d == 10 and i + 1 < 6 and (i + 1 < 3) == (i < 3):
                expect.add((a_key[(i + 1, j)], bi))
            if d == -10 and i - 1 >= 0 and (i - 1 < 3) == (i < 3):
                expect.add((a_key[(i - 1, j)], bi))
        got = list(zip(pa.tolist(), pb.tolist()))
        assert got == sorted(expect)


def test_candidate_pairs_requires_sorted_tiles():
    A = W.from_rings([rect(0, 0, 2, 2), rect(0, 0, 2, 2)], [1, 0])
    _, m = O.polygon_areas(A.off, A.xy)
    with pytest.raises(ValueError):
        O.candidate_pairs(m, A.tile, m, A.tile)


# ------------------------------------------------------------------------------- Jaccard

def test_jaccard_exact_rationals(cfg1):
    w = cfg1
    r = O.cross_compare(w.A, w.B)
    inter, uni = r["inter"], r["uni"]
    nz = inter > 0
    J = r["jaccard"]
    # J is the correctly rounded quotient of the two exact integer sums
    assert J["J"] == float(Fraction(int(inter[nz].sum()), int(uni[nz].sum())))
    # J' is the exact sum of the correctly rounded per-pair ratios, rounded once, divided by n
    exact = sum(Fraction(float(a) / float(b)) for a, b in zip(inter[nz].tolist(), uni[nz].tolist()))
    n = int(nz.sum())
    assert J["n_nonzero"] == n
    assert J["Jprime"] == float(exact) / n
    assert 0.3 < J["J"] < 1.0 and 0.3 < J["Jprime"] < 1.0


def test_jaccard_of_a_set_with_itself_is_one():
    """With pairwise MBR-disjoint polygons, each polygon's only candidate is itself: J = J' = 1."""
    rings = [[[30 * i, 0], [30 * i + 12, 2], [30 * i + 5, 17]] for i in range(20)]
    A = W.from_rings(rings)
    r = O.cross_compare(A, A)
    assert r["pa"].tolist() == list(range(20)) and r["pb"].tolist() == list(range(20))
    assert r["jaccard"]["J"] == 1.0 and r["jaccard"]["Jprime"] == 1.0


def test_jaccard_pairs_with_zero_intersection_are_excluded():
    inter = np.array([0, 3, 0, 5])
    uni = np.array([7, 6, 9, 10])
    J = O.jaccard(inter, uni)
    assert J["n_nonzero"] == 2 and J["sum_inter"] == 8 and J["sum_union"] == 16
    assert J["J"] == 0.5 and J["Jprime"] == 0.5
    assert O.jaccard(np.zeros(3, np.int64), np.ones(3, np.int64))["J"] == 0.0


# ------------------------------------------------------------------ other operators (Sec. 3.4)

SQ = [[0, 0], [4, 0], [4, 4], [0, 4]]


@pytest.mark.parametrize("other,expect", [
    ([[4, 0], [8, 0], [8, 4], [4, 4]], True),      # shared edge
    ([[4, 4], [8, 4], [8, 8], [4, 8]], True),      # shared corner only
    ([[4, 2], [7, 0], [7, 4]], True),              # a vertex on an edge
    ([[2, 2], [6, 2], [6, 6], [2, 6]], False),     # overlap: edges cross
    ([[1, 1], [2, 1], [2, 2], [1, 2]], False),     # inside: vertices within
    ([[5, 0], [8, 0], [8, 4], [5, 4]], False),     # disjoint
    ([[2, -1], [3, -1], [3, 5], [2, 5]], False),   # a strip through: edges cross
])
def test_touches_hand_cases(other, expect):
    assert O.touches(SQ, other) is expect
    assert O.touches(other, SQ) is expect


def test_touches_rectangles_closed_form():
    """Axis-aligned rectangles, closed form of the stated rule. Geometrically they touch when their
    closed boxes meet and their interiors do not (overlaps in x and y >= 0, one of them 0). The rule
    as stated also reports a touch when the interiors overlap but no corner of either lies strictly
    inside the other and no edges cross properly, which for rectangles happens exactly when their
    x-ranges or their y-ranges are equal (e.g. one inside the other along two shared edges)."""
    rng = np.random.Generator(np.random.PCG64(31))
    for _ in range(600):
        a = np.sort(rng.integers(0, 12, 2)); b = np.sort(rng.integers(0, 12, 2))
        c = np.sort(rng.integers(0, 12, 2)); d = np.sort(rng.integers(0, 12, 2))
        if a[0] == a[1] or b[0] == b[1] or c[0] == c[1] or d[0] == d[1]:
            continue
        p = [[a[0], b[0]], [a[1], b[0]], [a[1], b[1]], [a[0], b[1]]]
        q = [[c[0], d[0]], [c[1], d[0]], [c[1], d[1]], [c[0], d[1]]]
        ox = min(a[1], c[1]) - max(a[0], c[0])
        oy = min(b[1], d[1]) - max(b[0], d[0])
        geometric = ox >= 0 and oy >= 0 and (ox == 0 or oy == 0)
        same_range = (a[0] == c[0] and a[1] == c[1]) or (b[0] == d[0] and b[1] == d[1])
        expect = geometric or (ox > 0 and oy > 0 and same_range)
        assert O.touches(p, q) is bool(expect), (p, q)


def test_touches_symmetric_and_translation_invariant():
    rng = np.random.Generator(np.random.PCG64(32))
    x, y, c = W.star_rings(rng, rng.uniform(0, 60, 40), rng.uniform(0, 60, 40), rng.uniform(8, 30, 40),
                           rng.integers(3, 12, 40))
    off = np.concatenate([[0], np.cumsum(c)])
    rings = [np.stack([x[off[i]:off[i + 1]], y[off[i]:off[i + 1]]], 1) for i in range(40)]
    for i in range(0, 40, 2):
        p, q = rings[i], rings[i + 1]
        t = O.touches(p, q)
        assert O.touches(q, p) == t
        assert O.touches(p + [17, -5], q + [17, -5]) == t


def test_contains_flags_rectangles():
    """ST_Contains from areas: rectangle q inside rectangle p (closed form) <=> ||p n q|| = ||q||."""
    ra = [[[0, 0], [10, 0], [10, 10], [0, 10]], [[20, 0], [24, 0], [24, 4], [20, 4]]]
    rb = [[[2, 2], [5, 2], [5, 7], [2, 7]], [[8, 8], [12, 8], [12, 12], [8, 12]], [[20, 0], [24, 0], [24, 4], [20, 4]],
          [[-5, -5], [30, -5], [30, 30], [-5, 30]]]
    A, B = W.from_rings(ra), W.from_rings(rb)
    area_a, _ = O.polygon_areas(A.off, A.xy)
    area_b, _ = O.polygon_areas(B.off, B.xy)
    pa = np.array([0, 0, 1, 0, 1]); pb = np.array([0, 1, 2, 3, 3])
    inter, _ = O.pair_areas(A, B, pa, pb)
    f = O.contains_flags(area_a, area_b, pa, pb, inter)
    assert list(f) == [1, 0, 3, 2, 2]


# ------------------------------------------------------------------------------- membership masks

@pytest.mark.parametrize("method", ["brute", "rle"])
def test_mask_of_rectangles_and_triangles_closed_forms(method):
    """A rectangle's window is all inside; the right triangle (0,0), (n,0), (0,n) holds pixel (x, y)
    exactly when its centre is strictly below the hypotenuse, x + y + 1 < n: a centre on that edge
    does not count it, and the ray then meets no other edge. Its mirror image (0,0), (0,n), (-n,0)
    keeps the centres on its hypotenuse: the ray from such a centre does not count that edge but
    still crosses the edge x = 0, so pixel (x, y) is inside exactly when x + n >= y."""
    rng = np.random.default_rng(5)
    for _ in range(50):
        x0, y0 = (int(v) for v in rng.integers(-500, 500, 2))
        w, h = (int(v) for v in rng.integers(1, 70, 2))
        m = O.polygon_mask(rect(x0, y0, w, h), method)
        assert m.shape == (h, w) and m.all()
    for n in (1, 2, 3, 17, 64, 65, 100):
        m = O.polygon_mask([[0, 0], [n, 0], [0, n]], method)
        y, x = np.mgrid[0:n, 0:n]
        np.testing.assert_array_equal(m, x + y + 1 < n)
        mm = O.polygon_mask([[0, 0], [0, n], [-n, 0]], method)
        np.testing.assert_array_equal(mm, x >= y)          # column index x stands for pixel x - n
        assert mm.sum() == n * (n + 1) // 2


def test_masks_agree_with_each_other_the_pixel_test_and_the_areas():
    """The two mask methods are independent; each mask's popcount is the polygon's area and each of
    its cells is the per-pixel test."""
    w = W.single_tile(seed=9, n=60)
    rng = np.random.default_rng(3)
    for i in range(w.A.n):
        ring = w.A.xy[2 * w.A.off[i]: 2 * w.A.off[i + 1]].reshape(-1, 2)
        mb = O.polygon_mask(ring, "brute")
        np.testing.assert_array_equal(mb, O.polygon_mask(ring, "rle"))
        assert mb.sum() == O.polygon_area(ring) == O.polygon_area_rle(ring)
        x0, y0 = ring[:, 0].min(), ring[:, 1].min()
        for _ in range(5):
            yy, xx = int(rng.integers(0, mb.shape[0])), int(rng.integers(0, mb.shape[1]))
            assert mb[yy, xx] == bool(O.pixel_in_polygon(ring, x0 + xx, y0 + yy))
