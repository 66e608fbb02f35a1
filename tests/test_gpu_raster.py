"""GPU parity of the pixel rasters a prepared set keeps in device memory, and of the pair areas the
library computes from them (the AND of two rasters over a pair's window), against the CPU oracle.

Every membership bit, area and pair count is an integer: comparisons are exact (tolerance 0)."""
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


def rings_workload(rings_a, rings_b, tiles_a=None, tiles_b=None):
    return W.Workload("rings", W.from_rings(rings_a, tiles_a), W.from_rings(rings_b, tiles_b), 1, 0, 0)


def ring(ps, i):
    return ps.xy[2 * ps.off[i]: 2 * ps.off[i + 1]].reshape(-1, 2)


def decode_rasters(d):
    """(word offsets [n + 1], words, mbr [n, 4]) of a prepared set's raster buffer."""
    n = d.n
    buf = d.raster.cpu().numpy()[: int(d.c.raster_bytes)]
    hb = (8 * (n + 1) + 15) & ~15
    off = buf[: 8 * (n + 1)].view(np.int64)
    words = buf[hb:].view(np.uint32)
    assert off[n] == words.size
    return off, words, d.mbr.cpu().numpy()[:n]


def raster_bits(off, words, mbr, i):
    """Membership [H, W] of polygon i from its raster; also checks the padding bits are clear."""
    x0, y0, x1, y1 = (int(v) for v in mbr[i])
    Wd, H = x1 - x0, y1 - y0
    if Wd <= 0 or H <= 0:
        return np.zeros((max(H, 0), max(Wd, 0)), dtype=bool)
    nw = (Wd + 31) // 32
    if Wd <= 64 and H <= 64:
        assert off[i] == 128 * i                    # the polygon's slot
    else:
        assert off[i] >= 128 * len(mbr) and off[i] + H * nw <= words.size
    w = np.ascontiguousarray(words[off[i]: off[i] + H * nw]).reshape(H, nw)
    bits = np.unpackbits(w.view(np.uint8).reshape(H, nw, 4), axis=2, bitorder="little").reshape(H, 32 * nw)
    assert not bits[:, Wd:].any(), f"bits beyond the window of polygon {i}"
    return bits[:, :Wd].astype(bool)


def check_rasters(d, ps, brute_max=40_000):
    """Every polygon's raster against the oracle's membership mask (brute force for windows up to
    brute_max pixels, row intervals above) and its area against the mask's count."""
    off, words, mbr = decode_rasters(d)
    area = d.area.cpu().numpy()[: ps.n]
    for i in range(ps.n):
        r = ring(ps, i)
        x0, y0, x1, y1 = mbr[i]
        method = "brute" if (x1 - x0) * (y1 - y0) <= brute_max else "rle"
        want = O.polygon_mask(r, method)
        got = raster_bits(off, words, mbr, i)
        assert got.shape == want.shape, i
        if not np.array_equal(got, want):
            yy, xx = np.nonzero(got != want)
            raise AssertionError(f"polygon {i}: {len(yy)} pixels differ, first at row {yy[0]} col {xx[0]}")
        assert area[i] == want.sum(), i


def pair_run(ctx, w, mode, form="areas"):
    import paper_1208_0277_gb300 as P
    A, B = ctx.upload(w.A), ctx.upload(w.B)
    assert A.raster is not None and B.raster is not None
    pa, pb, tpo = ctx.candidate_pairs(A, B, with_tile_offsets=True)
    if form == "tiles":
        inter, uni = ctx.pair_areas_tiles(A, B, pa, pb, tpo)
    elif form == "batch":
        n = pa.numel()
        inter = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        uni = torch.empty_like(inter)
        res = torch.zeros(48, dtype=torch.uint8, device="cuda")
        ctx.batch_run(A, B, pa, pb, (inter[:n], uni[:n]), res)
        inter, uni = inter[:n], uni[:n]
    else:
        inter, uni = ctx.pair_areas(A, B, pa, pb, mode=mode)
    torch.cuda.synchronize()
    return A, B, pa.cpu().numpy().astype(np.int64), pb.cpu().numpy().astype(np.int64), \
        inter.cpu().numpy(), uni.cpu().numpy()


def oracle_pairs(w):
    """The oracle's candidate pairs (from its own MBRs)."""
    _, mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")
    return O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)


def edge_rings():
    """Windows of every size class the raster writers treat differently: 1..64 px (one or two words
    per row, written by the leaf), 65 px and more (difference rows), exactly 32 k px (the overflow
    word of a piece), 1024, 1025, 2048 and 2049 px wide (one to three 1024-column pieces), thin and tall, zero
    height or width (no words), repeated vertices, a self-intersecting ring, steep spikes, and
    negative coordinates."""
    rs = []
    for s in (1, 2, 31, 32, 33, 63, 64, 65, 96, 97, 128, 200):
        rs.append([[-s, 5], [0, 5], [0, 5 + s], [-s, 5 + s]])                        # square
        rs.append([[0, 0], [s, 0], [0, s]])                                           # triangles
        rs.append([[0, 0], [0, s], [-s, 0]])
        h = s // 2 + 1
        rs.append([[h, 0], [s + 1, h], [h, s + 1], [0, h]])                          # diamond
    rs.append([[0, 0], [2048, 0], [2048, 3], [1024, 40], [0, 3]])
    rs.append([[0, 0], [1024, 0], [1024, 30], [512, 77], [0, 30]])
    rs.append([[0, 0], [1025, 5], [1025, 9], [3, 66]])
    rs.append([[0, 0], [2049, 7], [2049, 9], [3, 45]])
    rs.append([[-1000, -1000], [3100, -990], [3096, -950], [-998, -951]])
    rs.append([[0, 0], [5, 0], [10, 0]])                                              # collinear: H = 0
    rs.append([[3, -20], [3, 30], [3, 10]])                                           # W = 0
    rs.append([[0, 0], [0, 0], [6, 0], [6, 0], [6, 5], [0, 5], [0, 5]])
    rs.append([[0, 0], [80, 80], [80, 0], [0, 80]])                                   # bow tie
    rs.append([[0, 0], [90, 1], [0, 2], [90, 3], [0, 4], [90, 5], [0, 6]])           # spikes
    teeth = 50
    comb = [[0, 0], [2 * teeth, 0]]
    for k in range(teeth - 1, -1, -1):
        comb += [[2 * k + 1, 3], [2 * k + 1, 70], [2 * k, 70]] + ([[2 * k, 3]] if k else [])
    rs.append(comb)
    return [np.asarray(r) for r in rs]


# ------------------------------------------------------------------------------- the rasters

def test_rasters_of_edge_case_windows(ctx):
    rs = edge_rings()
    w = rings_workload(rs, rs)
    check_rasters(ctx.upload(w.A), w.A)


def test_rasters_of_stars_medium_polygons_and_tissue(ctx):
    """Random nuclei, 60-600 px stars with up to 512 vertices (windows over 64 px: difference rows
    from the whole ring) and tissue regions with 1,024 or more vertices (band index: each 32-row band
    drawn from its own edge list)."""
    w = W.single_tile(seed=2, n=300)
    check_rasters(ctx.upload(w.A), w.A)
    rng = np.random.Generator(np.random.PCG64(7))
    n = 40
    x, y, c = W.star_rings(rng, rng.uniform(0, 3000, n), rng.uniform(0, 3000, n), rng.uniform(30.0, 300.0, n),
                           rng.integers(3, 513, n))
    off = np.concatenate([[0], np.cumsum(c)]).astype(np.int64)
    xy = np.empty(2 * x.shape[0], dtype=np.int32)
    xy[0::2], xy[1::2] = x, y
    ps = W.PolySet(off, xy, np.zeros(n, dtype=np.int32))
    check_rasters(ctx.upload(ps), ps)
    h = W.heavy_tail(seed=3, n_tiles=1, nuclei_per_tile=200, tissue_lo=3, tissue_hi=3, tissue_nv_lo=1024,
                     tissue_nv_hi=3000, tissue_s_lo=200.0, tissue_s_hi=900.0)
    d = ctx.upload(h.A)
    assert d.bands is not None
    check_rasters(d, h.A)
    # band lists wider than one 2048-column piece: zigzag tops of 1,101 vertices over 2,500 and 4,200 px
    rs = []
    for wdt, top in ((2500, 100), (4200, 70)):
        zig = [[int(k * wdt / 1100), top - 10 * (k % 2)] for k in range(1101)]
        rs.append(np.asarray([[0, 0], [wdt, -3]] + zig[::-1]))
    ps = W.from_rings(rs)
    d = ctx.upload(ps)
    assert d.bands is not None
    check_rasters(d, ps)


def test_raster_areas_equal_the_non_raster_prepare(ctx):
    """||p|| from rasters equals ||p|| from the other prepare paths on an uneven tile with polygons
    of every size, and the MBRs are the same."""
    w = W.subset_tiles(W.batched_uneven(seed=1, n_tiles=20), [0, 1, 2, 3])
    a = ctx.upload(w.A)
    b = ctx.upload(w.A, raster=False)
    np.testing.assert_array_equal(a.area.cpu().numpy(), b.area.cpu().numpy())
    np.testing.assert_array_equal(a.mbr.cpu().numpy(), b.mbr.cpu().numpy())
    want, mbr = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    np.testing.assert_array_equal(a.area.cpu().numpy()[: w.A.n], want)


# ------------------------------------------------------------------------------- pair areas

@pytest.mark.parametrize("form,mode", [("areas", 0), ("areas", 1), ("tiles", 0), ("batch", 1)])
def test_raster_pair_areas_match_oracle(ctx, form, mode):
    """Nuclei of one tile, the edge-case windows against each other (empty and one-pixel
    overlaps), and uneven tiles with polygons up to 400 px: every pair against the oracle."""
    rs = edge_rings()
    cases = [W.single_tile(seed=6, n=500),
             rings_workload(rs, [r + np.array([3, -2]) for r in rs] + rs[::-1]),
             W.subset_tiles(W.batched_uneven(seed=2, n_tiles=40), [0, 5, 7, 11])]
    for w in cases:
        A, B, pa, pb, inter, uni = pair_run(ctx, w, mode, form)
        ref_pa, ref_pb = oracle_pairs(w)
        np.testing.assert_array_equal(pa, ref_pa)
        np.testing.assert_array_equal(pb, ref_pb)
        ri, ru = O.pair_areas(w.A, w.B, ref_pa, ref_pb, method="rle")
        np.testing.assert_array_equal(inter, ri)
        np.testing.assert_array_equal(uni, ru)
    idx = np.arange(0, len(ref_pa), max(1, len(ref_pa) // 200))
    bi, bu = O.pair_areas(w.A, w.B, ref_pa[idx], ref_pb[idx], method="brute")
    np.testing.assert_array_equal(inter[idx], bi)
    np.testing.assert_array_equal(uni[idx], bu)


@pytest.mark.parametrize("heavy", [-1, 0, 1, 64, 1024, 1 << 30])
def test_raster_heavy_threshold_and_switch_keep_results(sccg, heavy):
    """Whether a pair is done by one warp or one CTA (raster_heavy), and whether rasters are used at
    all (rasters = 0), change nothing: tissue and nuclei of the heavy-tail workload, persistent form."""
    w = W.heavy_tail(seed=5, n_tiles=1, nuclei_per_tile=1500, tissue_lo=3, tissue_hi=4, tissue_nv_lo=500,
                     tissue_nv_hi=2500, tissue_s_lo=300.0, tissue_s_hi=1500.0)
    c = sccg.Context(0, {"raster_heavy": heavy})
    A, B, pa, pb, inter, uni = pair_run(c, w, 1)
    c.set_param("rasters", 0)
    i0, u0 = c.pair_areas(A, B, torch.from_numpy(pa.astype(np.int32)).cuda(),
                          torch.from_numpy(pb.astype(np.int32)).cuda(), mode=1)
    np.testing.assert_array_equal(inter, i0.cpu().numpy())
    np.testing.assert_array_equal(uni, u0.cpu().numpy())
    if heavy == 1024:
        ref_pa, ref_pb = oracle_pairs(w)
        np.testing.assert_array_equal(pa, ref_pa)
        np.testing.assert_array_equal(pb, ref_pb)
        ri, ru = O.pair_areas(w.A, w.B, ref_pa, ref_pb, method="rle")
        np.testing.assert_array_equal(inter, ri)
        np.testing.assert_array_equal(uni, ru)


@pytest.mark.parametrize("lanes", [1, 8, 16, 32])
def test_raster_lanes_per_pair_keep_results(sccg, lanes):
    """1, 8, 16 or 32 lanes per light pair (the pair's rows spread over its lane group): the same
    results as the oracle on nuclei and on uneven tiles with polygons up to 400 px."""
    c = sccg.Context(0, {"raster_lanes": lanes})
    for w in (W.single_tile(seed=12, n=700), W.subset_tiles(W.batched_uneven(seed=4, n_tiles=30), [1, 2, 9])):
        for mode in (0, 1):
            A, B, pa, pb, inter, uni = pair_run(c, w, mode)
            ref_pa, ref_pb = oracle_pairs(w)
            np.testing.assert_array_equal(pa, ref_pa)
            np.testing.assert_array_equal(pb, ref_pb)
            ri, ru = O.pair_areas(w.A, w.B, ref_pa, ref_pb, method="rle")
            np.testing.assert_array_equal(inter, ri)
            np.testing.assert_array_equal(uni, ru)


def test_raster_pairs_with_invalid_indices(ctx):
    """Out-of-range pair indices give -1 and leave the other pairs exact (raster path, both forms)."""
    w = W.single_tile(seed=8, n=200)
    A, B = ctx.upload(w.A), ctx.upload(w.B)
    _, mbr_a = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    _, mbr_b = O.polygon_areas(w.B.off, w.B.xy, method="rle")
    ref_pa, ref_pb = O.candidate_pairs(mbr_a, w.A.tile, mbr_b, w.B.tile)
    ri, ru = O.pair_areas(w.A, w.B, ref_pa, ref_pb, method="rle")
    pa = torch.from_numpy(ref_pa.astype(np.int32)).cuda()
    pb = torch.from_numpy(ref_pb.astype(np.int32)).cuda()
    bad = torch.tensor([0, 5, 17], device="cuda")
    pa[bad[:2]] = -1
    pb[bad[2]] = B.n
    for mode in (0, 1):
        inter, uni = ctx.pair_areas(A, B, pa, pb, mode=mode)
        inter, uni = inter.cpu().numpy(), uni.cpu().numpy()
        ok = np.ones(len(inter), dtype=bool)
        ok[bad.cpu().numpy()] = False
        assert (inter[~ok] == -1).all() and (uni[~ok] == -1).all()
        np.testing.assert_array_equal(inter[ok], ri[ok])
        np.testing.assert_array_equal(uni[ok], ru[ok])


# ------------------------------------------------------------------------------- buffers and sizing

def test_raster_buffer_too_small_falls_back_and_sizes_agree(sccg, ctx):
    """Through the C ABI: sccg_raster_bytes gives the size sccg_prepare reports; a buffer one byte
    short (or smaller than the offsets) leaves raster_ok 0 and the set prepared as without rasters
    (same areas; pair areas exact); the Python binding then allocates one of the exact size."""
    P = sccg
    w = W.subset_tiles(W.batched_uneven(seed=3, n_tiles=20), [0, 1])
    off = torch.from_numpy(w.A.off).cuda()
    xy = torch.from_numpy(w.A.xy).cuda()
    tile = torch.from_numpy(w.A.tile).cuda()
    n = w.A.n
    mbr = torch.empty((n, 4), dtype=torch.int32, device="cuda")
    area = torch.empty(n, dtype=torch.int64, device="cuda")
    c = P._native.PolySetC(n=n, off=off.data_ptr(), xy=xy.data_ptr(), tile=tile.data_ptr(), mbr=mbr.data_ptr(),
                           area=area.data_ptr())
    need = ctx.raster_bytes(c)
    want_area, _ = O.polygon_areas(w.A.off, w.A.xy, method="rle")
    for cap in (16, need - 1, need):
        buf = torch.zeros(max(cap, 16), dtype=torch.uint8, device="cuda")
        c.raster, c.raster_cap = buf.data_ptr(), cap
        assert ctx.lib.sccg_prepare(ctx.h, ctypes.byref(c), None) == 0
        assert c.raster_bytes == need
        assert c.raster_ok == (1 if cap >= need else 0)
        np.testing.assert_array_equal(area.cpu().numpy(), want_area)
    small = torch.zeros(64, dtype=torch.uint8, device="cuda")
    d = ctx.prepare(off, xy, tile, out=(mbr, area, small))
    assert d.raster is not None and d.raster.numel() == need and d.c.raster_ok == 1
    check_rasters(d, w.A)


def test_raster_prepare_rejects_invalid_sets_and_takes_empty_ones(ctx, sccg):
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [1, 1]]]))
    assert e.value.status == 1
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [16385, 0], [0, 3]]]))
    assert e.value.status == 2
    with pytest.raises(sccg.SccgError) as e:
        ctx.upload(W.from_rings([[[0, 0], [3, 0], [0, 3]], [[0, 0], [3, 0], [0, 3]]], tiles=[1, 0]))
    assert e.value.status == 1
    E = ctx.prepare(torch.zeros(1, dtype=torch.int64, device="cuda"),
                    torch.zeros(0, dtype=torch.int32, device="cuda"), None)
    assert E.n == 0
    A = ctx.upload(W.from_rings([[[0, 0], [3, 0], [0, 3]]]))
    pa, pb = ctx.candidate_pairs(A, E)
    assert pa.numel() == 0


def test_raster_prepare_sets_matches_single_prepares(ctx):
    specs, singles = [], []
    for seed in range(3):
        w = W.single_tile(seed=20 + seed, n=150)
        for P_ in (w.A, w.B):
            specs.append((torch.from_numpy(P_.off).cuda(), torch.from_numpy(P_.xy).cuda(),
                          torch.from_numpy(P_.tile).cuda(), None))
            singles.append(P_)
    many = ctx.prepare_sets(specs)
    for d, P_ in zip(many, singles):
        one = ctx.upload(P_)
        assert d.c.raster_ok == 1 and d.c.raster_bytes == one.c.raster_bytes
        # every polygon's raster (the unused parts of slots and the order of large rasters are free)
        da, db = decode_rasters(d), decode_rasters(one)
        np.testing.assert_array_equal(da[2], db[2])
        for i in range(P_.n):
            np.testing.assert_array_equal(raster_bits(*da, i), raster_bits(*db, i))
        np.testing.assert_array_equal(d.area.cpu().numpy(), one.area.cpu().numpy())
