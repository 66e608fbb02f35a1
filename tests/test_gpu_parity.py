"""GPU parity: the CUDA path through the C ABI against the CPU oracle, element by element.

Areas, MBRs, pair lists and the Jaccard values are integers or fixed doubles, so every comparison
is exact (tolerance 0)."""
import ctypes

import numpy as np
import pytest

import oracle as O
from paper_1208_0277_gb300 import workload as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sccg():
    import paper_1208_0277_gb300 as P
    P.build()
    return P


@pytest.fixture(scope="module")
def ctx(sccg):
    return sccg.Context(0)


def gpu_run(ctx, w, mode=0):
    import paper_1208_0277_gb300 as P
    A = ctx.upload(w.A, raster=False)
    B = ctx.upload(w.B, raster=False)
    r = P.cross_compare(ctx, A, B, mode=mode)
    torch.cuda.synchronize()
    return dict(area_a=A.area.cpu().numpy()[: w.A.n], area_b=B.area.cpu().numpy()[: w.B.n],
                mbr_a=A.mbr.cpu().numpy()[: w.A.n], mbr_b=B.mbr.cpu().numpy()[: w.B.n],
                pa=r["pa"].cpu().numpy().astype(np.int64), pb=r["pb"].cpu().numpy().astype(np.int64),
                inter=r["inter"].cpu().numpy(), uni=r["uni"].cpu().numpy(), jaccard=r["jaccard"])


def assert_same(g, ref):
    np.testing.assert_array_equal(g["mbr_a"], ref["mbr_a"])
    np.testing.assert_array_equal(g["mbr_b"], ref["mbr_b"])
    np.testing.assert_array_equal(g["area_a"], ref["area_a"])
    np.testing.assert_array_equal(g["area_b"], ref["area_b"])
    np.testing.assert_array_equal(g["pa"], ref["pa"])
    np.testing.assert_array_equal(g["pb"], ref["pb"])
    np.testing.assert_array_equal(g["inter"], ref["inter"])
    np.testing.assert_array_equal(g["uni"], ref["uni"])
    for k in ("sum_inter", "sum_union", "n_nonzero", "J", "Jprime"):
        assert g["jaccard"][k] == ref["jaccard"][k], k


# ------------------------------------------------------------------------------- workloads

def test_single_tile_bit_exact(ctx):
    w = W.single_tile(seed=0)
    assert_same(gpu_run(ctx, w), O.cross_compare(w.A, w.B))


@pytest.mark.parametrize("words", [1, 0])
@pytest.mark.parametrize("T", [2, 33, 200, 1024, 4096, 8192, 1 << 22])
def test_threshold_does_not_change_results(sccg, T, words):
    """T only decides where subdivision stops (Sec. 3.4) and leaf_words how a leaf is pixelized;
    results must be identical for every setting."""
    w = W.single_tile(seed=3, n=400)
    c = sccg.Context(0, {"T": T, "area_T": T, "leaf_words": words})
    assert_same(gpu_run(c, w), O.cross_compare(w.A, w.B))


@pytest.mark.parametrize("wpc", [1, 3, 8])
def test_warps_per_cta(sccg, wpc):
    w = W.single_tile(seed=4, n=300)
    c = sccg.Context(0, {"warps_per_cta": wpc, "T": 64})
    assert_same(gpu_run(c, w), O.cross_compare(w.A, w.B))


def medium_polygons(seed, n=60, s_lo=60.0, s_hi=300.0, nv_hi=300, kind="nucleus"):
    rng = np.random.Generator(np.random.PCG64(seed))
    cx = rng.uniform(0, 1500, n)
    cy = rng.uniform(-800, 700, n)
    s = rng.uniform(s_lo, s_hi, n)
    nv = rng.integers(3, nv_hi + 1, n)
    x, y, c = W.star_rings(rng, cx, cy, s, nv, kind)
    off = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(c, out=off[1:])
    xy = np.empty(2 * x.shape[0], dtype=np.int32)
    xy[0::2], xy[1::2] = x, y
    return W.PolySet(off, xy, np.zeros(n, dtype=np.int32))


@pytest.mark.parametrize("T", [2, 64, 512, 4096])
def test_medium_and_large_polygons_subdivision_and_chunked_edges(sccg, T):
    """Windows of 60..300 px (several subdivision levels) and up to 300 vertices (edge buffers
    re-staged chunk by chunk); concave 'tissue' rings as well."""
    A = medium_polygons(10)
    B = medium_polygons(11, kind="tissue")
    w = W.Workload("medium", A, B, 1, 2048, 0)
    for words in (1, 0):
        c = sccg.Context(0, {"T": T, "area_T": T, "leaf_words": words})
        g = gpu_run(c, w)
        ref = O.cross_compare(A, B, method="rle")
        assert_same(g, ref)
    idx = np.arange(0, len(ref["pa"]), max(1, len(ref["pa"]) // 25))
    bi, bu = O.pair_areas(A, B, ref["pa"][idx], ref["pb"][idx], method="brute")
    np.testing.assert_array_equal(g["inter"][idx], bi)
    np.testing.assert_array_equal(g["uni"][idx], bu)


def test_whole_slide_tiles_sampled(ctx):
    """Several tiles of the whole-slide workload: every pair against the row-interval oracle and a
    sample against the brute force."""
    w = W.subset_tiles(W.whole_slide(seed=0), [0, 1, 26, 312, 624])
    g = gpu_run(ctx, w)
    ref = O.cross_compare(w.A, w.B, method="rle")
    assert_same(g, ref)
    rng = np.random.default_rng(0)
    idx = rng.choice(len(ref["pa"]), 2000, replace=False)
    bi, bu = O.pair_areas(w.A, w.B, ref["pa"][idx], ref["pb"][idx], method="brute")
    np.testing.assert_array_equal(g["inter"][idx], bi)
    np.testing.assert_array_equal(g["uni"][idx], bu)


def test_tile_pair_offsets_and_one_launch_per_tile(ctx):
    w = W.subset_tiles(W.whole_slide(seed=0), [3, 4, 5, 30, 31])
    A, B = ctx.upload(w.A, raster=False), ctx.upload(w.B, raster=False)
    pa, pb, tpo = ctx.candidate_pairs(A, B, with_tile_offsets=True)
    pa_h = pa.cpu().numpy()
    assert tpo[0] == 0 and tpo[-1] == len(pa_h)
    for t in range(5):
        assert np.all(w.A.tile[pa_h[tpo[t]:tpo[t + 1]]] == t)
    before = ctx.launch_count()
    inter, uni = ctx.pair_areas_tiles(A, B, pa, pb, tpo)
    torch.cuda.synchronize()
    assert ctx.launch_count() - before == int((np.diff(tpo) > 0).sum())
    i2, u2 = ctx.pair_areas(A, B, pa, pb)
    np.testing.assert_array_equal(inter.cpu().numpy(), i2.cpu().numpy())
    np.testing.assert_array_equal(uni.cpu().numpy(), u2.cpu().numpy())
    _, mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")
    opa, opb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    np.testing.assert_array_equal(pa_h, opa)
    np.testing.assert_array_equal(pb.cpu().numpy(), opb)
    ref_i, ref_u = O.pair_areas(w.A, w.B, opa, opb, method="rle")
    np.testing.assert_array_equal(inter.cpu().numpy(), ref_i)
    np.testing.assert_array_equal(uni.cpu().numpy(), ref_u)


@pytest.mark.parametrize("split,T", [(32, 256), (100, 256), (4096, 256), (4096, 8192), (900, 1 << 22)])
def test_persistent_queue_matches_oracle(sccg, split, T):
    """Persistent form: one launch, device work queue, windows cut into items of about `split`
    pixels (many items per pair for small `split`); results identical to the oracle. Items of
    fewer than T pixels are single leaves and stream their edges (k_pair_areas_stream); larger
    ones are staged and subdivided (k_pair_areas_persistent and its overflow levels)."""
    c = sccg.Context(0, {"split_pixels": split, "T": T})
    w = W.single_tile(seed=5, n=500)
    assert_same(gpu_run(c, w, mode=1), O.cross_compare(w.A, w.B))
    A = medium_polygons(12)
    B = medium_polygons(13, kind="tissue")
    wm = W.Workload("medium", A, B, 1, 2048, 0)
    assert_same(gpu_run(c, wm, mode=1), O.cross_compare(A, B, method="rle"))


def leaf_case_rings(seed):
    """Pairs whose windows are exactly 1, 2, 31, 32, 33, 63 and 64 pixels wide and high (rectangles,
    and triangles and diamonds with steep edges and centres on diagonals inside such windows), pairs
    with touching MBRs (empty windows, no work items) between them, and random stars."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ra, rb = [], []
    x = 0
    for s in (1, 2, 31, 32, 33, 63, 64, 64, 33, 32):
        for _ in range(3):
            dx, dy = int(rng.integers(1, 9)), int(rng.integers(1, 9))
            ra.append([[x, 0], [x + s + dx, 0], [x + s + dx, s + dy], [x, s + dy]])
            rb.append([[x + dx, dy], [x + dx + s, dy], [x + dx + s, dy + s], [x + dx, dy + s]])
            # touching MBRs: the window is one column wide and empty of pixels
            ra.append([[x, 200], [x + 10, 200], [x + 10, 210], [x, 210]])
            rb.append([[x + 10, 200], [x + 20, 205], [x + 10, 210]])
            # a steep triangle (edges spanning up to s rows) against a diamond, both in one window
            ra.append([[x, 300], [x + s // 2 + 1, 300 + s], [x + s + 1, 300]])
            h = s // 2 + 1
            rb.append([[x + h, 300], [x + s + 1, 300 + h], [x + h, 300 + s + 1], [x, 300 + h]])
            x += s + 20
    cx = rng.uniform(0, x, 200)
    cy = rng.uniform(400, 600, 200)
    sz = rng.uniform(10.0, 70.0, 200)
    nv = rng.integers(3, 80, 200)
    xs, ys, c = W.star_rings(rng, cx, cy, sz, nv)
    st = np.concatenate([[0], np.cumsum(c)])
    stars = [np.stack([xs[st[i]:st[i + 1]], ys[st[i]:st[i + 1]]], 1) for i in range(200)]
    ra += [r for r in stars[:100]]
    rb += [r + rng.integers(-4, 5, 2) for r in stars[:100]]
    rb += [r for r in stars[100:]]
    return [np.asarray(r) for r in ra], [np.asarray(r) for r in rb]


@pytest.mark.parametrize("lanes", [32, 1])
@pytest.mark.parametrize("split", [4096, 1024, 300])
def test_leaf_items_window_sizes_steep_edges_and_empty_pairs(sccg, split, lanes):
    """The leaf form of the persistent queue (items of at most 64 x 64 pixels, one leaf each, both
    rings streamed as one edge sequence): windows of 1 to 64 pixels a side (one or two 32-pixel halves
    per row), edges spanning many rows (their crossings spread over the lanes), pairs without items
    between pairs with items, and over 32 pairs per queue take (the per-warp pair table is refilled);
    side 64 and smaller sides that cut windows into several items; with one warp per item, and with
    small pairs (windows up to 32 x 32, up to 64 edges) one lane each. Against the oracle."""
    c = sccg.Context(0, {"split_pixels": split, "T": 8192, "pair_lanes": lanes})
    ra, rb = leaf_case_rings(31)
    w = rings_workload(ra, rb)
    assert_same(gpu_run(c, w, mode=1), O.cross_compare(w.A, w.B))


@pytest.mark.parametrize("mode", [0, 1])
def test_heavy_tail_tissue_and_nuclei(sccg, mode):
    """Tissue polygons (500-2000 vertices, 400-1200 px) among nuclei: large A polygons take the
    bitmap path of the candidate-pair join, edges are re-staged chunk by chunk, windows are deeply
    subdivided; the persistent form cuts the big windows into many items."""
    w = W.heavy_tail(seed=2, n_tiles=2, nuclei_per_tile=1500, tissue_lo=3, tissue_hi=4, tissue_nv_lo=500,
                     tissue_nv_hi=2000, tissue_s_lo=400.0, tissue_s_hi=1200.0)
    c = sccg.Context(0, {"split_pixels": 20000})
    g = gpu_run(c, w, mode=mode)
    ref = O.cross_compare(w.A, w.B, method="rle")
    assert_same(g, ref)
    idx = np.arange(0, len(ref["pa"]), max(1, len(ref["pa"]) // 300))
    bi, bu = O.pair_areas(w.A, w.B, ref["pa"][idx], ref["pb"][idx], method="brute")
    np.testing.assert_array_equal(g["inter"][idx], bi)
    np.testing.assert_array_equal(g["uni"][idx], bu)


@pytest.mark.parametrize("mode,T", [(0, 64), (1, 64), (1, 8192)])
def test_band_index_gives_the_same_results(sccg, mode, T):
    """Polygons with >= 1024 vertices get a band index; items then stage only their bands' edges.
    Concave tissue rings and rectilinear staircases (horizontal edges on band boundaries) against
    nuclei, with small work items in the persistent form so item windows start at many offsets
    relative to the bands: identical to the run without the index and to the oracle."""
    w = W.heavy_tail(seed=3, n_tiles=1, nuclei_per_tile=800, tissue_lo=3, tissue_hi=3, tissue_nv_lo=1024,
                     tissue_nv_hi=3000, tissue_s_lo=200.0, tissue_s_hi=600.0)
    rng = np.random.Generator(np.random.PCG64(21))
    stairs, _ = W.staircase_rings(rng, 4, max_cols=700, max_h=60, origin_span=300)
    small, _ = W.staircase_rings(rng, 300, max_cols=12, max_h=15, origin_span=600)
    ws = rings_workload([np.asarray(r) for r in stairs] + [np.asarray(r) for r in small],
                        [np.asarray(r) for r in small] + [np.asarray(r) for r in stairs])
    c = sccg.Context(0, {"split_pixels": 400, "T": T})     # T = 8192: items stream their bands' records
    for wk in (w, ws):
        with_bands = gpu_run(c, wk, mode=mode)
        A, B = c.upload(wk.A, bands=False, raster=False), c.upload(wk.B, bands=False, raster=False)
        assert A.bands is None
        import paper_1208_0277_gb300 as P
        r = P.cross_compare(c, A, B, mode=mode)
        np.testing.assert_array_equal(with_bands["inter"], r["inter"].cpu().numpy())
        np.testing.assert_array_equal(with_bands["uni"], r["uni"].cpu().numpy())
        ref = O.cross_compare(wk.A, wk.B, method="rle")
        assert_same(with_bands, ref)
    assert c.upload(w.A, raster=False).bands is not None


def test_heavy_tail_full_size_tissue(sccg):
    """One tile of the heavy-tail workload at full tissue size (2,000-20,000 vertices, MBR up to
    4,000 px, with band indexes) among 3,000 nuclei: areas and candidate pairs against the oracle in
    full, pair areas (persistent form) on every tissue-tissue pair and a seeded sample of the
    others (the oracle's row-interval method; its brute force would take hours here)."""
    w = W.heavy_tail(seed=4, n_tiles=1, nuclei_per_tile=3000, tissue_lo=4, tissue_hi=5)
    c = sccg.Context(0)
    A, B = c.upload(w.A, raster=False), c.upload(w.B, raster=False)
    assert A.bands is not None and B.bands is not None
    mbrs = []
    for P_, d in ((w.A, A), (w.B, B)):
        ref_area, ref_mbr = O.polygon_areas(P_.off, P_.xy, method="rle")
        np.testing.assert_array_equal(d.area.cpu().numpy()[: P_.n], ref_area)
        np.testing.assert_array_equal(d.mbr.cpu().numpy()[: P_.n], ref_mbr)
        mbrs.append(ref_mbr)
    pa, pb = c.candidate_pairs(A, B)
    opa, opb = O.candidate_pairs(mbrs[0], w.A.tile, mbrs[1], w.B.tile)
    np.testing.assert_array_equal(pa.cpu().numpy(), opa)
    np.testing.assert_array_equal(pb.cpu().numpy(), opb)
    inter, uni = c.pair_areas(A, B, pa, pb, mode=1)
    torch.cuda.synchronize()
    big_a = np.diff(w.A.off)[opa] >= 1000
    big_b = np.diff(w.B.off)[opb] >= 1000
    rng = np.random.Generator(np.random.PCG64(9))
    both = np.nonzero(big_a & big_b)[0]
    one = np.nonzero(big_a ^ big_b)[0]
    none = np.nonzero(~big_a & ~big_b)[0]
    idx = np.sort(np.concatenate([both, rng.choice(one, min(150, len(one)), replace=False),
                                  rng.choice(none, min(3000, len(none)), replace=False)]))
    assert len(both) > 0 and len(one) > 0
    ri, ru = O.pair_areas(w.A, w.B, opa[idx], opb[idx], method="rle")
    np.testing.assert_array_equal(inter.cpu().numpy()[idx], ri)
    np.testing.assert_array_equal(uni.cpu().numpy()[idx], ru)


@pytest.mark.parametrize("T", [2, 256, 8192, 1 << 28])
def test_nosep_variant_counts_the_union_directly(sccg, T):
    """PixelBox-NoSep (Sec. 5.2): the union counted by subdivision of the union window equals the
    oracle's directly counted union; T = 2^28 is PixelOnly. Nuclei, concave polygons, staircases."""
    c = sccg.Context(0, {"T": T})
    rng = np.random.Generator(np.random.PCG64(8))
    ra, _ = W.staircase_rings(rng, 60, max_cols=30, max_h=30, origin_span=60)
    rb, _ = W.staircase_rings(rng, 60, max_cols=30, max_h=30, origin_span=60)
    for wk, meth in ((W.single_tile(seed=3, n=400), "brute"),
                     (W.Workload("medium", medium_polygons(14, n=40), medium_polygons(15, n=40, kind="tissue"),
                                 1, 2048, 0), "rle"),
                     (rings_workload([np.asarray(r) for r in ra], [np.asarray(r) for r in rb]), "brute")):
        assert_same(gpu_run(c, wk, mode=sccg.MODE_NOSEP), O.cross_compare(wk.A, wk.B, method=meth))


def test_nosep_refuses_wide_polygons(sccg):
    c = sccg.Context(0)
    w = rings_workload([[[0, 0], [9000, 0], [0, 40]]], [[[0, 0], [50, 0], [0, 50]]])
    A, B = c.upload(w.A, raster=False), c.upload(w.B, raster=False)
    pa, pb = c.candidate_pairs(A, B)
    with pytest.raises(sccg.SccgError) as e:
        c.pair_areas(A, B, pa, pb, mode=sccg.MODE_NOSEP)
    assert e.value.status == 2


@pytest.mark.parametrize("mode", [0, 1])
def test_a_20000_vertex_polygon(sccg, mode):
    """A rectilinear staircase of about 24,000 vertices (6,600 one-pixel columns) against small
    polygons along it and against a shifted copy of itself: area, pairs and areas by the band index,
    right-side culling and the overflow path, against the oracle's row-interval method."""
    rng = np.random.Generator(np.random.PCG64(41))
    big, heights = W.staircase_rings(rng, 1, max_cols=10_000, max_h=6, origin_span=1)
    big = np.asarray(big[0])
    assert len(big) >= 15_000
    small, _ = W.staircase_rings(rng, 300, max_cols=12, max_h=12, origin_span=1)
    shift = rng.integers(0, 9_000, 300)
    small = [np.asarray(r) + [int(s), 0] for r, s in zip(small, shift)]
    w = rings_workload([big] + small[:150], [big + [3, 1]] + small[150:])
    c = sccg.Context(0, {"split_pixels": 1024})
    g = gpu_run(c, w, mode=mode)
    ref = O.cross_compare(w.A, w.B, method="rle")
    assert_same(g, ref)
    assert g["area_a"][0] == int(heights[0].sum())


def test_batch_graph_replay_and_recapture(sccg):
    """sccg_batch_run: persistent areas + Jaccard captured once as a CUDA graph and replayed; a new
    pair list (other buffers) triggers a new capture. Results equal the oracle every time."""
    c = sccg.Context(0, {"split_pixels": 64})
    for seed in (6, 7):
        w = W.single_tile(seed=seed, n=500)
        A, B = c.upload(w.A, raster=False), c.upload(w.B, raster=False)
        pa, pb = c.candidate_pairs(A, B)
        inter = torch.full((pa.numel(),), -7, dtype=torch.int64, device="cuda")
        uni = torch.full_like(inter, -7)
        res = torch.zeros(48, dtype=torch.uint8, device="cuda")
        ref = O.cross_compare(w.A, w.B)
        for _ in range(2):
            inter.fill_(-7)
            c.batch_run(A, B, pa, pb, (inter, uni), res)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(inter.cpu().numpy(), ref["inter"])
            np.testing.assert_array_equal(uni.cpu().numpy(), ref["uni"])
            J = c.read_jaccard(res)
            for k in ("sum_inter", "sum_union", "n_nonzero", "J", "Jprime"):
                assert J[k] == ref["jaccard"][k], k


def test_batch_graph_with_large_polygons(sccg):
    """The graph form when polygons exceed 64 vertices: the big queue runs on the side stream (fork and
    join inside the captured graph) with 128-edge buffers and the overflow kernel; replayed twice."""
    c = sccg.Context(0, {"split_pixels": 256})
    A_, B_ = medium_polygons(16, n=50), medium_polygons(17, n=50, kind="tissue")
    A, B = c.upload(A_, raster=False), c.upload(B_, raster=False)
    pa, pb = c.candidate_pairs(A, B)
    inter = torch.full((pa.numel(),), -7, dtype=torch.int64, device="cuda")
    uni = torch.full_like(inter, -7)
    res = torch.zeros(48, dtype=torch.uint8, device="cuda")
    ref = O.cross_compare(A_, B_, method="rle")
    for _ in range(2):
        inter.fill_(-7)
        c.batch_run(A, B, pa, pb, (inter, uni), res)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(inter.cpu().numpy(), ref["inter"])
        np.testing.assert_array_equal(uni.cpu().numpy(), ref["uni"])
        J = c.read_jaccard(res)
        for k in ("sum_inter", "sum_union", "n_nonzero", "J", "Jprime"):
            assert J[k] == ref["jaccard"][k], k


# ------------------------------------------------------------------------------- edge cases

def rings_workload(rings_a, rings_b):
    return W.Workload("rings", W.from_rings(rings_a), W.from_rings(rings_b), 1, 0, 0)


def test_edge_cases_ties_degenerate_selfintersecting(ctx):
    tri = [[0, 0], [4, 0], [0, 4]]
    tri2 = [[0, 0], [4, 0], [4, 4]]
    tri3 = [[0, 0], [4, 4], [0, 4]]
    diamond = [[2, 0], [4, 2], [2, 4], [0, 2]]
    collinear = [[0, 0], [5, 0], [10, 0]]                 # zero area, zero-height window
    thin = [[0, 0], [10, 0], [10, 1], [0, 1]]             # 1-row window
    tall = [[3, -20], [4, -20], [4, 30], [3, 30]]         # 1-column window
    dup = [[0, 0], [0, 0], [6, 0], [6, 0], [6, 5], [0, 5], [0, 5]]   # repeated vertices
    bowtie = [[0, 0], [8, 8], [8, 0], [0, 8]]             # self-intersecting ring (even-odd)
    spike = [[0, 0], [9, 1], [0, 2], [9, 3], [0, 4], [9, 5], [0, 6]]  # centres on many edges
    rect_stack = [[1, 1], [7, 1], [7, 7], [1, 7]]
    # 30 teeth: every row of the 40-row window is crossed 60 times (too many for the per-row edge
    # lists of one band, so the window falls back to the general leaf path)
    comb = [[0, 0]] + [p for k in range(30) for p in ([2 * k + 1, 40], [2 * k + 2, 0])] + [[60, -1], [0, -1]]
    comb_cover = [[-2, -3], [63, -3], [63, 45], [-2, 45]]
    rings = [tri, tri2, tri3, diamond, collinear, thin, tall, dup, bowtie, spike, rect_stack, comb, comb_cover]
    w = rings_workload(rings, rings[::-1])
    assert_same(gpu_run(ctx, w), O.cross_compare(w.A, w.B))


def comb_ring(teeth, h=40):
    """A bar with `teeth` one-pixel teeth: each row through the teeth is crossed 2 * teeth times."""
    pts = [[0, 0], [2 * teeth, 0]]
    for k in range(teeth - 1, -1, -1):
        pts += [[2 * k + 1, 3], [2 * k + 1, h], [2 * k, h]] + ([[2 * k, 3]] if k else [])
    return pts


@pytest.mark.parametrize("area_T", [65536, 64])
@pytest.mark.parametrize("method", [0, 1])
def test_polygon_area_methods_match_oracle(sccg, method, area_T):
    """||p|| by rows (default) and by PixelBox on the polygon alone, on shapes that stress each:
    rows crossed by more edges than one pass holds (combs of 520 and 700 teeth), self-intersecting
    random rings, concave tissue polygons, staircases and ties."""
    rng = np.random.Generator(np.random.PCG64(11))
    stairs, _ = W.staircase_rings(rng, 80, max_cols=40, max_h=30)
    selfx = [rng.integers(0, 60, size=(int(rng.integers(3, 300)), 2)).tolist() for _ in range(40)]
    ties = [[[0, 0], [4, 2], [0, 4]], [[0, 0], [2, 2], [4, 0]], [[0, 0], [4, 4], [0, 8], [-4, 4]]]
    rings = [comb_ring(700), comb_ring(520, 9), comb_ring(30)] + selfx + ties + [np.asarray(r).tolist() for r in stairs]
    sets = [W.from_rings(rings), medium_polygons(12, n=40, kind="tissue"), W.single_tile(seed=5, n=400).A]
    ctx = sccg.Context(0, {"area_method": method, "area_T": area_T})
    for P in sets:
        d = ctx.upload(P, raster=False)
        torch.cuda.synchronize()
        ref, _ = O.polygon_areas(P.off, P.xy, method="rle")
        np.testing.assert_array_equal(d.area.cpu().numpy()[: P.n], ref)


def test_rectilinear_staircases_match_shoelace(ctx):
    rng = np.random.Generator(np.random.PCG64(7))
    rings, heights = W.staircase_rings(rng, 200, max_cols=40, max_h=30)
    w = rings_workload(rings, rings)
    g = gpu_run(ctx, w)
    np.testing.assert_array_equal(g["area_a"], [int(h.sum()) for h in heights])
    assert_same(g, O.cross_compare(w.A, w.B))


def test_shoelace_areas_of_rectilinear_sets(sccg):
    """area_method SHOELACE (Sec. 3.2's closed form for sets flagged rectilinear and simple): the
    staircases' areas come from their shoelace sums and equal the oracle's pixel counts (and the
    column sums); star polygons mixed into the set have diagonal edges and are counted by pixels;
    the pair areas and unions that use these areas match the oracle."""
    rng = np.random.Generator(np.random.PCG64(8))
    rings, heights = W.staircase_rings(rng, 300, max_cols=60, max_h=40)
    stars = [np.asarray(r) for r in leaf_case_rings(5)[0][-40:]]
    w = rings_workload(rings + stars, stars + rings)
    c = sccg.Context(0, {"area_method": sccg.AREA_SHOELACE})
    g = gpu_run(c, w, mode=1)
    np.testing.assert_array_equal(g["area_a"][: len(rings)], [int(h.sum()) for h in heights])
    assert_same(g, O.cross_compare(w.A, w.B))


def test_coordinate_and_extent_limits(ctx):
    L = 1 << 28
    big = [[L - 16384, L - 5], [L, L - 5], [L, L], [L - 16384, L]]            # extent exactly 16384
    neg = [[-L, -L], [-L + 300, -L + 7], [-L + 11, -L + 290]]
    diag = [[0, 0], [16384, 1], [1, 16384]]                                    # 16384^2 window
    w = rings_workload([big, neg, diag], [big, neg, [[5, 5], [16000, 40], [30, 16200]]])
    g = gpu_run(ctx, w)
    ref = O.cross_compare(w.A, w.B, method="rle")
    assert_same(g, ref)


def test_empty_sets_and_no_pairs(ctx):
    w = rings_workload([[[0, 0], [3, 0], [0, 3]]], [[[10, 10], [13, 10], [10, 13]]])
    g = gpu_run(ctx, w)
    assert len(g["pa"]) == 0
    assert g["jaccard"]["n_nonzero"] == 0 and g["jaccard"]["J"] == 0.0
    import paper_1208_0277_gb300 as P
    E = ctx.prepare(torch.zeros(1, dtype=torch.int64, device="cuda"),
                    torch.zeros(0, dtype=torch.int32, device="cuda"), None, raster=False)
    pa, pb = ctx.candidate_pairs(E, E)
    assert pa.numel() == 0
    assert P.cross_compare(ctx, E, E)["jaccard"]["n_pairs"] == 0


def test_prepare_sets_matches_single_prepares(ctx, sccg):
    """sccg_prepare_sets: several sets with one synchronisation, the same MBRs, areas and summaries
    as one call per set; a set that fails validation is reported and left unprepared."""
    w = W.single_tile(seed=4, n=300)
    dev = torch.device("cuda")
    specs = [(torch.from_numpy(P_.off).to(dev), torch.from_numpy(P_.xy).to(dev), torch.from_numpy(P_.tile).to(dev),
              None) for P_ in (w.A, w.B, w.A)]
    many = ctx.prepare_sets(specs, raster=False)
    for d, P_ in zip(many, (w.A, w.B, w.A)):
        one = ctx.upload(P_, raster=False)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(d.area.cpu().numpy(), one.area.cpu().numpy())
        np.testing.assert_array_equal(d.mbr.cpu().numpy(), one.mbr.cpu().numpy())
        assert (d.c.max_nv, d.c.max_extent, d.c.n_tiles) == (one.c.max_nv, one.c.max_extent, one.c.n_tiles)
        assert d.c.reserved == one.c.reserved
    bad = W.from_rings([[[0, 0], [1, 1]]])
    specs.insert(1, (torch.from_numpy(bad.off).to(dev), torch.from_numpy(bad.xy).to(dev), None, None))
    with pytest.raises(sccg.SccgError) as e:
        ctx.prepare_sets(specs, raster=False)
    assert e.value.status == 1


# ------------------------------------------------------------------------------- errors

def test_invalid_inputs_rejected_on_the_host(ctx, sccg):
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [1, 1]]]), raster=False)
    assert e.value.status == 1
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [16385, 0], [0, 3]]]), raster=False)
    assert e.value.status == 2
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [3, 0], [0, 3]], [[0, 0], [3, 0], [0, 3]]], tiles=[1, 0]), raster=False)
    assert e.value.status == 1
    # a host pointer where device memory is required
    A = ctx.upload(W.from_rings([[[0, 0], [3, 0], [0, 3]]]), raster=False)
    host = np.zeros(4, dtype=np.int64)
    st = ctx.lib.sccg_pair_areas(ctx.h, ctypes.byref(A.c), ctypes.byref(A.c), host.ctypes.data,
                                 host.ctypes.data, 1, host.ctypes.data, host.ctypes.data, 0, None)
    assert st == 1


@pytest.mark.parametrize("kind", ["single", "heavy"])
def test_candidate_pairs_speculative_sizes(sccg, kind):
    """The candidate-pair grid's buffers sized before their counts are known (default), from the
    counts (two more synchronisations), or too small on purpose (the call notices and redoes itself
    with exact sizes): the same pairs, in the same order, with the same tile offsets, as the oracle."""
    if kind == "single":
        w = W.single_tile(seed=8, n=700)
    else:
        w = W.heavy_tail(seed=4, n_tiles=2, nuclei_per_tile=1200, tissue_lo=3, tissue_hi=4, tissue_nv_lo=300,
                         tissue_nv_hi=900, tissue_s_lo=300.0, tissue_s_hi=900.0)
    mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")[1]
    mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")[1]
    ref_pa, ref_pb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    got = []
    for mode in (1, 0, 2, 1):
        c = sccg.Context(0)
        c.set_param("candidate_speculative", mode)
        A, B = c.upload(w.A, raster=False), c.upload(w.B, raster=False)
        pa, pb, tpo = c.candidate_pairs(A, B, with_tile_offsets=True)
        got.append((pa.cpu().numpy(), pb.cpu().numpy(), np.asarray(tpo)))
        c.close()
    for pa, pb, tpo in got:
        np.testing.assert_array_equal(pa, ref_pa)
        np.testing.assert_array_equal(pb, ref_pb)
        np.testing.assert_array_equal(tpo, got[0][2])


@pytest.mark.parametrize("area_T", [8192, 600])
def test_prepare_leaf_and_rows_boundaries(sccg, area_T):
    """Polygon areas around the limits of k_prepare's paths (one leaf of parity rows for boxes up to
    64 x 64 px under area_T pixels, streamed parity words above 64 px, rows from area_T on): boxes 31 to
    33 px a side, 4 to 129 vertices, rings with collinear runs, boxes on both sides of area_T; also the
    polygons of at most 128 vertices alone and the others alone."""
    rng = np.random.Generator(np.random.PCG64(17))
    rings = []
    for side in (31, 32, 33):
        for nv in (4, 127, 128, 129):
            t = np.sort(rng.uniform(0, 2 * np.pi, nv))
            x = np.rint(100 * len(rings) + side / 2 + (side / 2) * np.cos(t))
            y = np.rint(side / 2 + (side / 2) * np.sin(t))
            rings.append(np.stack([x, y], 1).astype(np.int64))
        # a rectangle whose edges run along its box, with extra collinear vertices
        x0 = 100 * len(rings)
        rings.append(np.array([[x0, 0], [x0 + side // 2, 0], [x0 + side, 0], [x0 + side, side], [x0, side]]))
    import paper_1208_0277_gb300 as P
    c = P.Context(0, {"area_T": area_T})
    for sel in (rings, [r for r in rings if len(r) <= 128], [r for r in rings if len(r) > 128]):
        ps = W.from_rings([np.asarray(r) for r in sel])
        d = c.upload(ps, raster=False)
        torch.cuda.synchronize()
        ref_area, ref_mbr = O.polygon_areas(ps.off, ps.xy)
        np.testing.assert_array_equal(d.area.cpu().numpy()[: ps.n], ref_area)
        np.testing.assert_array_equal(d.mbr.cpu().numpy()[: ps.n], ref_mbr)


def test_full_density_uneven_tile(sccg):
    """One tile of the 2,000-uneven-tiles workload at its densest (20,000 polygons per set, MBR
    lognormal 8-400 px, 4-512 vertices), through the persistent form with the default parameters:
    every MBR, polygon area, candidate pair and pair area against the oracle (its O(n m) pairs and
    exact row-interval areas), element by element."""
    w = W.batched_uneven(seed=11, n_tiles=1, count_lo=20_000, count_hi=20_000)
    assert w.A.n == 20_000
    c = sccg.Context(0)
    assert_same(gpu_run(c, w, mode=1), O.cross_compare(w.A, w.B, method="rle"))


def test_jaccard_ratios_are_the_ieee_quotients(ctx):
    """Each ratio inter/union summed into J' is the IEEE double quotient (the library forms it in
    integers): with one pair per segment, a segment's J' is that ratio alone. Quotients of every
    magnitude from 2^-31 to 1, equal operands, powers of two and their neighbours, against numpy's
    division; the whole set's J and J' against the oracle."""
    rng = np.random.default_rng(17)
    u = np.concatenate([
        rng.integers(1, 200, 20000), rng.integers(1, 1 << 16, 20000), rng.integers(1 << 20, 1 << 31, 40000),
        np.array([(1 << k) + d for k in range(1, 31) for d in (-1, 0, 1)]), np.full(1000, (1 << 31) - 1)])
    frac = rng.random(u.size)
    i = np.maximum(1, (frac * u).astype(np.int64))
    i[:500] = u[:500]                               # ratio 1
    i[500:1000] = 1                                 # the smallest ratios
    i = np.minimum(i, u).astype(np.int64)
    u = u.astype(np.int64)
    inter, uni = torch.from_numpy(i).cuda(), torch.from_numpy(u).cuda()
    seg = torch.arange(i.size + 1, dtype=torch.int64, device="cuda")
    out = torch.zeros(48 * i.size, dtype=torch.uint8, device="cuda")
    ctx.jaccard_segments(inter, uni, seg, out)
    got = np.array([r["Jprime"] for r in ctx.decode_jaccard_array(out.cpu().numpy())])
    want = i.astype(np.float64) / u.astype(np.float64)
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, (i[bad[:5]], u[bad[:5]], got[bad[:5]], want[bad[:5]])
    ref = O.jaccard(i, u)
    res = ctx.jaccard(inter, uni)
    for k in ("sum_inter", "sum_union", "n_nonzero", "J", "Jprime"):
        assert res[k] == ref[k], k
