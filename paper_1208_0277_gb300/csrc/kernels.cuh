// Kernels of the cross-comparison path: set preparation (MBR + ||p||), candidate pairs (filter),
// pair areas (aggregator, plain and persistent forms) and the Jaccard reduction.
#pragma once
#include <cstdint>

#include "leaf64.cuh"
#include "pixelbox.cuh"
#include "scanline.cuh"

// Dynamic shared memory of the one-warp-per-item kernels (per-warp WarpSmem slices).
#ifndef SCCG_DYNAMIC_SMEM
#define SCCG_DYNAMIC_SMEM(T, name) extern __shared__ T name[]
#endif

// Minimum resident CTAs per SM requested from the compiler for the one-warp-per-item kernels
// (0: no request). 4 CTAs of 256 threads cap registers at 64 (32 resident warps per SM).
#ifndef SCCG_MIN_BLOCKS
#define SCCG_MIN_BLOCKS 4
#endif
#if SCCG_MIN_BLOCKS > 0
#define SCCG_ITEM_BOUNDS __launch_bounds__(256, SCCG_MIN_BLOCKS)
#else
#define SCCG_ITEM_BOUNDS __launch_bounds__(256)
#endif
// The kernels whose leaves stream their edges need little shared memory, so registers set their
// occupancy: at least 4 resident CTAs of 256 threads for k_prepare (64 registers: with its table of
// 32 polygons per warp, 10.75 ms for both prepares of the uneven tiles against 11.24 ms with 5 and
// 12.49 ms with 3) and 4 for k_pair_areas_stream (the heavy tail's large items; 6.6 against 7.4 ms
// with 6).
#ifndef SCCG_PREP_MIN_BLOCKS
#define SCCG_PREP_MIN_BLOCKS 4
#endif
#ifndef SCCG_STREAM_MIN_BLOCKS
#define SCCG_STREAM_MIN_BLOCKS 4
#endif
#ifndef SCCG_LEAF_MIN_BLOCKS
#define SCCG_LEAF_MIN_BLOCKS 4
#endif
#ifndef SCCG_LANE_MIN_BLOCKS
#define SCCG_LANE_MIN_BLOCKS 4
#endif

namespace sccg {

constexpr int kCoordLimit = 1 << 28;   // |x|, |y| <= 2^28
constexpr int kExtentLimit = 16384;    // bounding box width / height
constexpr int kMaxVertices = 1 << 24;

// error bits reported by the prepare kernel
constexpr int kErrFewVertices = 1;
constexpr int kErrRange = 2;
constexpr int kErrTiles = 4;

struct PrepStats {
    int err;
    int max_nv;
    int max_extent;
    int n_tiles;
    long long first_bad;
    unsigned long long band_bytes;    // sum of the band index block sizes
    unsigned deferred;                // polygons listed for a second kernel (area not yet written)
    unsigned next;                    // k_raster_big's claim counter over the listed polygons
    unsigned long long raster_words;  // words of the set's pixel rasters (sets that keep them)
    unsigned takes;                   // k_prepare's claim counter over the takes of 32 polygons
    unsigned pad;
};

__device__ __forceinline__ void flush_counters(WorkCounters* out, const WorkCounters& wc)
{
    const unsigned long long* in = &wc.strip_edges;
    unsigned long long* dst = &out->strip_edges;
    constexpr int kFields = sizeof(WorkCounters) / sizeof(unsigned long long);
#pragma unroll
    for (int k = 0; k < kFields; ++k) {
        unsigned long long v = in[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if ((threadIdx.x & 31) == 0) atomicAdd(dst + k, v);
    }
}

// ----------------------------------------------------------------------------------------------
// Band index of the polygons with many vertices. A polygon's pixel rows are cut into bands of
// 2^kBandShift rows counted from its minimum y; band b lists the edge record {ylo, dy, dx, xl} of
// every edge whose closed y-range [ylo, ylo + dy] meets the band's rows. A work item then stages
// only the records of the bands its window's rows fall in (stage_banded) instead of reading the
// whole ring.
//
// Blob (16-byte aligned): BandHead; int64 tab[n] (byte offset of polygon i's block, -1 = none);
// the blocks. Block: int nb and 3 pad ints; int boff[nb + 1] (exclusive offsets of the bands'
// lists) and int cur[nb] (fill cursors), padded to 16 bytes; int4 ent[boff[nb]].
// ----------------------------------------------------------------------------------------------
constexpr int kBandShift = 5;
static_assert((1 << kBandShift) <= 32, "a band's rows are counted one lane per row");
#ifndef SCCG_BAND_MIN_VERTICES
#define SCCG_BAND_MIN_VERTICES 1024
#endif
constexpr int kBandMinVertices = SCCG_BAND_MIN_VERTICES;
constexpr long long kBandMaxEntries = 1LL << 30;

struct BandHead {
    long long n;
    long long bytes;
    int shift;
    int pad[3];
};

__host__ __device__ inline long long band_head_bytes(long long n)
{
    return (long long)sizeof(BandHead) + ((8 * n + 15) & ~15LL);
}
__host__ __device__ inline long long band_block_bytes(int nb, long long entries)
{
    return 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL) + 16 * entries;
}

// Block size of polygon i (0 when it gets no index). Whole warp, converged.
__device__ __forceinline__ long long band_block_size(const int2* v, int nv, int miny, int maxy, int lane)
{
    if (nv < kBandMinVertices) return 0;
    const int nb = ((maxy - miny) >> kBandShift) + 1;
    long long entries = 0;
    for (int base = 0; base < nv; base += 32) {
        const int e = base + lane;
        if (e < nv) {
            const int f = (e + 1 == nv) ? 0 : e + 1;
            const int ya = v[e].y, yb = v[f].y;
            entries += (long long)(((max(ya, yb) - miny) >> kBandShift) - ((min(ya, yb) - miny) >> kBandShift) + 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) entries += __shfl_xor_sync(kFull, entries, o);
    return entries > kBandMaxEntries ? 0 : band_block_bytes(nb, entries);
}

// ----------------------------------------------------------------------------------------------
// a1 + a2: per-polygon MBR, validation and pixel area ||p||. One warp per polygon.
// ----------------------------------------------------------------------------------------------
// Per-warp shared memory of k_prepare's streamed areas: the XorRows of area_stream or the Leaf64 of
// leaf_area (the same bytes).
constexpr size_t kPrepWarpBytes = ((sizeof(XorRows) > sizeof(Leaf64) ? sizeof(XorRows) : sizeof(Leaf64)) + 15) &
                                  ~size_t(15);


struct PrepArgs {
    long long n;
    const int64_t* off;
    const int32_t* xy;
    const int32_t* tile;
    int4* mbr;
    int64_t* area;
    PrepStats* stats;
    int T;
    WorkCounters* counters;
    int defer_above;        // > 0: polygons with more vertices are listed for k_prepare_big
    int* big_list;
    unsigned* big_n;
    int words;              // as AreasArgs::words
    int shoelace;           // 1: ||p|| of a polygon whose edges are all axis-parallel from its shoelace sum
    // pixel rasters (RASTER): polygon i's words start at word rhead[i] of rwords; a window of at most
    // 64 x 64 pixels has the slot of kRasterSlot words at kRasterSlot * i (written here when rleaf),
    // larger ones are placed after the slots once their sizes are known (k_raster_place)
    long long* rhead;       // [n + 1]
    uint32_t* rwords;
    int rleaf;              // 1: the header and the slots fit the buffer
};

constexpr int kRasterSlot = 128;        // words of a leaf window's raster slot: 64 rows of 2 words

// Words of the pixel raster of a polygon whose window is W x H pixels: H rows of ceil(W / 32).
__host__ __device__ inline long long raster_words_of(int W, int H)
{
    return (W > 0 && H > 0) ? (long long)H * ((W + 31) >> 5) : 0;
}

// Sizing of a set's pixel rasters (sccg_raster_bytes): MBR, validation and, for every polygon whose
// window is over 64 pixels wide or high, its raster's word count (0 for the others, which take a
// fixed slot, and for invalid ones), one warp per polygon.
__global__ void __launch_bounds__(256, 8) k_mbr(const PrepArgs a, long long* words)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    int err = 0, max_nv = 0, max_ext = 0, max_tile = -1;
    long long first_bad = 0x7fffffffffffffffLL;
    long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    // a memory-bound pass: the next polygon's offsets are loaded while this one's vertices are read,
    // and each lane keeps four vertex loads in flight
    long long o0 = 0, o1 = 0;
    if (i < a.n) { o0 = a.off[i]; o1 = a.off[i + 1]; }
    for (; i < a.n; i += nwarps) {
        long long q0 = 0, q1 = 0;
        if (i + nwarps < a.n) { q0 = a.off[i + nwarps]; q1 = a.off[i + nwarps + 1]; }
        const long long nvl = o1 - o0;
        const int2* v = reinterpret_cast<const int2*>(a.xy) + o0;
        int e = 0;
        int x0 = 0x7fffffff, y0 = 0x7fffffff, x1 = -0x7fffffff, y1 = -0x7fffffff;
        if (nvl < 3 || nvl > kMaxVertices) {
            e = kErrFewVertices;
        } else {
            const int nv = (int)nvl;
            for (int base = 0; base < nv; base += 128) {
                int2 p[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int k = base + 32 * u + lane;
                    p[u] = k < nv ? v[k] : v[0];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    x0 = min(x0, p[u].x); x1 = max(x1, p[u].x);
                    y0 = min(y0, p[u].y); y1 = max(y1, p[u].y);
                }
            }
            x0 = __reduce_min_sync(kFull, x0); y0 = __reduce_min_sync(kFull, y0);
            x1 = __reduce_max_sync(kFull, x1); y1 = __reduce_max_sync(kFull, y1);
            if (x0 < -kCoordLimit || y0 < -kCoordLimit || x1 > kCoordLimit || y1 > kCoordLimit ||
                x1 - x0 > kExtentLimit || y1 - y0 > kExtentLimit)
                e = kErrRange;
        }
        int t = 0;
        if (a.tile) {
            t = a.tile[i];
            if (t < 0 || (i > 0 && a.tile[i - 1] > t)) e |= kErrTiles;
        }
        if (lane == 0) {
            a.mbr[i] = make_int4(x0, y0, x1, y1);
            words[i] = (e || (x1 - x0 <= 64 && y1 - y0 <= 64)) ? 0 : raster_words_of(x1 - x0, y1 - y0);
        }
        if (e) { err |= e; first_bad = min(first_bad, i); }
        max_nv = max(max_nv, (int)min(nvl, (long long)0x7fffffff));
        if (e == 0) max_ext = max(max_ext, max(x1 - x0, y1 - y0));
        max_tile = max(max_tile, t);
        o0 = q0;
        o1 = q1;
    }
    if (lane == 0) {
        if (err) { atomicOr(&a.stats->err, err); atomicMin(&a.stats->first_bad, first_bad); }
        atomicMax(&a.stats->max_nv, max_nv);
        atomicMax(&a.stats->max_extent, max_ext);
        atomicMax(&a.stats->n_tiles, max_tile + 1);
    }
}

// SCAN: a polygon whose window holds fewer than T pixels is pixelized here as one leaf, its edges
// streamed from the ring (PixelBox's one-leaf case, cheapest for small windows; shared memory per
// warp: one XorRows); every other one is listed for k_area_bands (by rows). Otherwise by PixelBox on
// the polygon alone (per-warp WarpSmem), deferring polygons with more than defer_above vertices to
// k_prepare_big.
//
// RASTER (sets that keep pixel rasters; SCAN only): a polygon whose window is at most 64 x 64 pixels
// is pixelized here as one leaf and its rows are written to its raster slot (when rleaf); every
// larger one is listed (its raster's words added to stats->raster_words) for k_raster_big, which
// writes both its raster and ||p|| once the listed rasters are placed, or for k_area_bands when they
// do not fit the buffer.
// The next take of k_prepare from its counter, for the whole warp. Whole warp, converged.
__device__ __forceinline__ long long claim_take(unsigned* takes, int lane)
{
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(takes, 1u);
    return (long long)__shfl_sync(kFull, t, 0);
}

template <int CAP, int STK, bool COUNT, bool SCAN, bool RASTER = false>
__global__ void __launch_bounds__(256, SCCG_PREP_MIN_BLOCKS) k_prepare(const PrepArgs a)
{
    static_assert(SCAN || !RASTER, "rasters are written by the streamed leaves");
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[SCAN ? 0 : warp];
    char* wbytes = reinterpret_cast<char*>(smem4) + (SCAN ? warp * kPrepWarpBytes : 0);
    XorRows& X = *reinterpret_cast<XorRows*>(wbytes);
    Leaf64& L = *reinterpret_cast<Leaf64*>(wbytes);      // small windows use the same per-warp bytes
    WorkCounters wc = {};
    unsigned long long big_words = 0;
    int err = 0, max_nv = 0, max_ext = 0, max_tile = -1;
    long long first_bad = 0x7fffffffffffffffLL;
    unsigned long long band_bytes = 0;
    if (RASTER && a.rleaf) {
        // leaf_area writing rasters keeps the leaf rows zero between polygons
        for (int k = lane; k < kLeafWords; k += 32) L.w[k] = 0u;
        __syncwarp();
    }
    // Each warp takes 32 consecutive polygons at a time (the next free take claimed from a counter, so
    // that warps whose takes hold small rings take more of them): lane j loads polygon j's offsets and
    // tile ids (coalesced), the warp pixelizes the 32 one after another, lane j keeps polygon j's
    // results, and the 32 MBRs, areas and raster offsets are stored together.
    const long long n_takes = (a.n + 31) / 32;
    for (long long tk = claim_take(&a.stats->takes, lane); tk < n_takes; tk = claim_take(&a.stats->takes, lane)) {
    const long long c0 = tk * 32;
    const long long ij = c0 + lane;
    long long oj0 = 0, oj1 = 0;
    int tj = 0;
    bool tbad = false;
    if (ij < a.n) {
        oj0 = a.off[ij];
        oj1 = a.off[ij + 1];
        if (a.tile) {
            tj = a.tile[ij];
            tbad = tj < 0 || (ij > 0 && a.tile[ij - 1] > tj);
        }
    }
    const int cnt = (int)min(32LL, a.n - c0);
    if (RASTER) {
        // the take's 32 rings are contiguous: their lines are requested into L2 now (at most 64 KB),
        // so that each polygon's vertex loads below wait on L2 rather than DRAM
        const long long v0 = __shfl_sync(kFull, oj0, 0), v1 = __shfl_sync(kFull, oj1, cnt - 1);
        const char* vb = reinterpret_cast<const char*>(a.xy) + 8 * v0;
        const long long nbytes = min(8 * (v1 - v0), 65536LL);
        for (long long o = 128LL * lane; o < nbytes; o += 32 * 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(vb + o));
    }
    int4 my_mbr = make_int4(0, 0, 0, 0);
    uint32_t my_area = 0;
    bool my_defer = false;
    int my_e = 0;
    for (int j = 0; j < cnt; ++j) {
        const long long i = c0 + j;
        const long long o0 = __shfl_sync(kFull, oj0, j), o1 = __shfl_sync(kFull, oj1, j);
        const long long nvl = o1 - o0;
        const int2* v = reinterpret_cast<const int2*>(a.xy) + o0;
        int e = 0;
        int x0 = 0x7fffffff, y0 = 0x7fffffff, x1 = -0x7fffffff, y1 = -0x7fffffff;
        if (nvl < 3 || nvl > kMaxVertices) {
            e = kErrFewVertices;
        } else {
            const int nv = (int)nvl;
            for (int base = 0; base < nv; base += 32) {
                const int k = base + lane;
                if (k < nv) {
                    const int2 p = v[k];
                    x0 = min(x0, p.x); x1 = max(x1, p.x);
                    y0 = min(y0, p.y); y1 = max(y1, p.y);
                }
            }
            x0 = warp_min(x0); y0 = warp_min(y0);
            x1 = warp_max(x1); y1 = warp_max(y1);
            if (x0 < -kCoordLimit || y0 < -kCoordLimit || x1 > kCoordLimit || y1 > kCoordLimit ||
                x1 - x0 > kExtentLimit || y1 - y0 > kExtentLimit)
                e = kErrRange;
        }
        uint32_t area = 0;
        // Rectilinear sets (Sec. 3.2's POLYAREA): when every edge of the ring is axis-parallel, ||p|| is
        // |twice the shoelace sum| / 2 (coordinates taken relative to the box corner, so every product
        // stays below 2^28 and the sum below 2^52); the caller's flag vouches that the ring is simple,
        // where this equals the pixel count. A ring with any other edge is counted by pixels below.
        bool closed_form = false;
        if (SCAN && !RASTER && a.shoelace && e == 0) {
            const int nv = (int)nvl;
            long long twice = 0;
            bool axis = true;
            for (int base = 0; base < nv; base += 32) {
                const int k = base + lane;
                if (k < nv) {
                    const int2 p = v[k];
                    const int2 q = v[k + 1 == nv ? 0 : k + 1];
                    axis &= (p.x == q.x) | (p.y == q.y);
                    twice += (long long)(p.x - x0) * (q.y - y0) - (long long)(q.x - x0) * (p.y - y0);
                }
            }
            axis = __all_sync(kFull, axis);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) twice += __shfl_xor_sync(kFull, twice, o);
            if (axis) {
                closed_form = true;
                area = (uint32_t)((twice < 0 ? -twice : twice) >> 1);
            }
        }
        // SCAN: a polygon whose window is not small is deferred to k_area_bands (by rows).
        // Otherwise the large ones to k_prepare_big.
        const bool leaf_win = x1 - x0 <= kLeafSide && y1 - y0 <= kLeafSide;
        const bool small_win = RASTER ? leaf_win : (long long)(x1 - x0) * (y1 - y0) < a.T;
        const bool by_rows = SCAN && !small_win;
        const bool defer = e == 0 && !closed_form && (by_rows || (!SCAN && a.defer_above > 0 && nvl > a.defer_above));
        if (lane == 0 && defer) a.big_list[atomicAdd(a.big_n, 1u)] = (int)i;
        if (RASTER && lane == 0 && defer) big_words += (unsigned long long)raster_words_of(x1 - x0, y1 - y0);
        if (SCAN && e == 0 && !defer && !closed_form && x1 > x0 && y1 > y0) {
            if (leaf_win) {
                // with rasters the leaf's parity rows are also the polygon's raster, written to its slot
                area = leaf_area<COUNT>(v, (int)nvl, x0, y0, x1, y1, L, lane, wc,
                                        RASTER && a.rleaf ? a.rwords + (long long)kRasterSlot * i : nullptr);
            } else {
                area = area_stream<COUNT>(v, (int)nvl, x0, y0, x1, y1, X, lane, wc);
            }
        } else if (!SCAN && e == 0 && !defer && x1 > x0 && y1 > y0) {
            const int nv = (int)nvl;
            const bool res = nv <= CAP;
            __syncwarp();
            if (res) stage_edges(v, nv, 0, nv, S.ep, S.rp, lane);
            __syncwarp();
            const PolyPair pp{v, nv, res, v, nv, res};
            area = pixelbox<false, COUNT>(pp, x0, y0, x1, y1, a.T, a.words, S, lane, wc);
        }
        if (e == 0) band_bytes += (unsigned long long)band_block_size(v, (int)nvl, y0, y1, lane);
        if (lane == j) {
            my_mbr = make_int4(x0, y0, x1, y1);
            my_area = area;
            my_defer = defer;
            my_e = e;
        }
    }
    if (ij < a.n) {
        const int e = my_e | (tbad ? kErrTiles : 0);
        a.mbr[ij] = my_mbr;
        if (!my_defer) a.area[ij] = (int64_t)my_area;
        if (RASTER && a.rleaf && !my_defer) a.rhead[ij] = (long long)kRasterSlot * ij;
        if (e) { err |= e; first_bad = min(first_bad, ij); }
        max_nv = max(max_nv, (int)min(oj1 - oj0, (long long)0x7fffffff));
        if (e == 0) max_ext = max(max_ext, max(my_mbr.z - my_mbr.x, my_mbr.w - my_mbr.y));
        max_tile = max(max_tile, tj);
    }
    }
    // the lanes' statistics, reduced over the warp
    err = (int)__reduce_or_sync(kFull, (unsigned)err);
    max_nv = __reduce_max_sync(kFull, max_nv);
    max_ext = __reduce_max_sync(kFull, max_ext);
    max_tile = __reduce_max_sync(kFull, max_tile);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) first_bad = min(first_bad, __shfl_xor_sync(kFull, first_bad, o));
    if (lane == 0) {
        if (err) { atomicOr(&a.stats->err, err); atomicMin(&a.stats->first_bad, first_bad); }
        atomicMax(&a.stats->max_nv, max_nv);
        atomicMax(&a.stats->max_extent, max_ext);
        atomicMax(&a.stats->n_tiles, max_tile + 1);
        if (band_bytes) atomicAdd(&a.stats->band_bytes, band_bytes);
        if (RASTER && big_words) atomicAdd(&a.stats->raster_words, big_words);
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// Areas of the polygons k_prepare listed (more than defer_above vertices), with larger edge
// buffers; their MBRs were written and validated by k_prepare.
template <int CAP, int STK, bool COUNT>
__global__ void SCCG_ITEM_BOUNDS k_prepare_big(const PrepArgs a)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[warp];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    WorkCounters wc = {};
    const long long nbig = *a.big_n;
    for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + warp; j < nbig; j += nwarps) {
        const long long i = a.big_list[j];
        const long long o0 = a.off[i];
        const int nv = (int)(a.off[i + 1] - o0);
        const int2* v = reinterpret_cast<const int2*>(a.xy) + o0;
        const int4 m = a.mbr[i];
        uint32_t area = 0;
        if (m.z > m.x && m.w > m.y) {
            const bool res = nv <= CAP;
            __syncwarp();
            if (res) stage_edges(v, nv, 0, nv, S.ep, S.rp, lane);
            __syncwarp();
            const PolyPair pp{v, nv, res, v, nv, res};
            area = pixelbox<false, COUNT>(pp, m.x, m.y, m.z, m.w, a.T, a.words, S, lane, wc);
        }
        if (lane == 0) a.area[i] = (int64_t)area;
    }
    if (COUNT) flush_counters(a.counters, wc);
}

__global__ void k_band_sizes(long long n, const int64_t* off, const int32_t* xy, const int4* mbr, long long* size)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const long long o0 = off[i];
        const int nv = (int)(off[i + 1] - o0);
        const int4 m = mbr[i];
        const long long s = band_block_size(reinterpret_cast<const int2*>(xy) + o0, nv, m.y, m.w, lane);
        if (lane == 0) size[i] = s;
    }
}

// tab[i] from the scanned block sizes; the header from one thread.
__global__ void k_band_tab(long long n, const long long* size, const long long* boffs, char* blob, long long bytes)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    long long* tab = reinterpret_cast<long long*>(blob + sizeof(BandHead));
    if (i == 0) {
        BandHead* h = reinterpret_cast<BandHead*>(blob);
        h->n = n;
        h->bytes = bytes;
        h->shift = kBandShift;
    }
    if (i < n) tab[i] = size[i] > 0 ? band_head_bytes(n) + boffs[i] : -1;
}

__global__ void k_band_fill(long long n, const int64_t* off, const int32_t* xy, const int4* mbr, char* blob)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long* tab = reinterpret_cast<const long long*>(blob + sizeof(BandHead));
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const long long at = tab[i];
        if (at < 0) continue;                       // warp-uniform
        const long long o0 = off[i];
        const int nv = (int)(off[i + 1] - o0);
        const int2* v = reinterpret_cast<const int2*>(xy) + o0;
        const int4 m = mbr[i];
        const int nb = ((m.w - m.y) >> kBandShift) + 1;
        int* head = reinterpret_cast<int*>(blob + at);
        int* boff = head + 4;
        int* cur = boff + nb + 1;
        int4* ent = reinterpret_cast<int4*>(blob + at + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
        if (lane == 0) head[0] = nb;
        for (int b = lane; b <= nb; b += 32) boff[b] = 0;
        __syncwarp();
        for (int base = 0; base < nv; base += 32) {
            const int e = base + lane;
            if (e < nv) {
                const int f = (e + 1 == nv) ? 0 : e + 1;
                const int ya = v[e].y, yb = v[f].y;
                const int b0 = (min(ya, yb) - m.y) >> kBandShift, b1 = (max(ya, yb) - m.y) >> kBandShift;
                for (int b = b0; b <= b1; ++b) atomicAdd(&boff[b], 1);
            }
        }
        __syncwarp();
        int carry = 0;
        for (int base = 0; base <= nb; base += 32) {       // exclusive scan, 32 bands at a time
            const int b = base + lane;
            const int c = b <= nb ? boff[b] : 0;
            int incl = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(kFull, incl, o);
                if (lane >= o) incl += t;
            }
            if (b <= nb) boff[b] = carry + incl - c;
            if (b < nb) cur[b] = 0;
            carry += __shfl_sync(kFull, incl, 31);
        }
        __syncwarp();
        for (int base = 0; base < nv; base += 32) {
            const int e = base + lane;
            if (e < nv) {
                const int f = (e + 1 == nv) ? 0 : e + 1;
                int2 a = v[e];
                int2 b = v[f];
                if (b.y < a.y) { const int2 t = a; a = b; b = t; }
                const int4 rec = make_int4(a.y, b.y - a.y, b.x - a.x, a.x);
                const int b0 = (a.y - m.y) >> kBandShift, b1 = (b.y - m.y) >> kBandShift;
                for (int bb = b0; bb <= b1; ++bb) ent[boff[bb] + atomicAdd(&cur[bb], 1)] = rec;
            }
        }
        __syncwarp();
    }
}

// ||p|| of the polygons k_prepare deferred (list[0 .. *n_list)), by rows: one warp per polygon,
// band by band. A polygon with a block in the band index (blob may be null) takes each band's rows
// from the edges listed for that band (band_rows), so no band rescans the whole ring; the others
// are counted from their rings (area_scan).
template <bool COUNT>
__global__ void SCCG_ITEM_BOUNDS k_area_bands(const int64_t* off, const int32_t* xy, const int4* mbr, const char* blob,
                                              const int* list, const unsigned* n_list, int64_t* area,
                                              WorkCounters* counters)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    ScanSmem& S = reinterpret_cast<ScanSmem*>(smem4)[warp];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    WorkCounters wc = {};
    const long long nl = *n_list;
    for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + warp; j < nl; j += nwarps) {
        const long long i = list[j];
        const long long o0 = off[i];
        const int nv = (int)(off[i + 1] - o0);
        const int2* v = reinterpret_cast<const int2*>(xy) + o0;
        const int4 m = mbr[i];
        uint32_t acc = 0;
        if (m.z > m.x && m.w > m.y) {
            const long long at = blob ? reinterpret_cast<const long long*>(blob + sizeof(BandHead))[i] : -1;
            if (at >= 0) {
                const char* blk = blob + at;
                const int nb = reinterpret_cast<const int*>(blk)[0];
                const int* boff = reinterpret_cast<const int*>(blk) + 4;
                const int4* ent = reinterpret_cast<const int4*>(blk + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
                for (int b = 0; b < nb; ++b) {
                    const int b0 = m.y + (b << kBandShift);
                    const int nrows = min(1 << kBandShift, m.w - b0);
                    if (nrows <= 0) break;
                    acc += band_rows<COUNT>(RecordEdges{ent + boff[b], boff[b + 1] - boff[b]}, b0, nrows, m.x, m.z,
                                            v, nv, S, lane, wc);
                }
                acc = warp_sum(acc);
            } else {
                acc = area_scan<COUNT>(v, nv, m.x, m.y, m.z, m.w, S, lane, wc);
            }
        }
        if (lane == 0) area[i] = (int64_t)acc;
    }
    if (COUNT) flush_counters(counters, wc);
}

// The records of polygon block `blk` (polygon min y `miny`) that stage_culled would keep for the
// window [x0, x1) x [y0, y1), read from the bands covering rows y0 .. y1 - 1 only. An edge listed
// in several of those bands is taken from the first of them. Same return convention as
// stage_culled. Whole warp, converged.
__device__ __forceinline__ int stage_banded(const char* blk, int miny, int x0, int y0, int x1, int y1, int4* E,
                                            float* R, int cap, int lane, bool right, unsigned long long& flip)
{
    const bool rows64 = right && y1 - y0 <= 64;
    unsigned long long fl = 0;
    const int* head = reinterpret_cast<const int*>(blk);
    const int nb = head[0];
    const int* boff = head + 4;
    const int4* ent = reinterpret_cast<const int4*>(blk + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
    const int b0 = min(max((y0 - miny) >> kBandShift, 0), nb - 1);
    const int b1 = min(max((y1 - 1 - miny) >> kBandShift, 0), nb - 1);
    int cnt = 0;
    for (int b = b0; b <= b1; ++b) {
        const int e0 = boff[b], e1 = boff[b + 1];
        for (int base = e0; base < e1; base += 32) {
            const int k = base + lane;
            bool keep = false;
            int4 rec = make_int4(0, 0, 0, 0);
            if (k < e1) {
                rec = ent[k];
                const int first = max(b0, (rec.x - miny) >> kBandShift);
                keep = (first == b) & (rec.x < y1) & (rec.x + rec.y > y0) & (max(rec.w, rec.w + rec.z) > x0);
                if (keep && rows64 && min(rec.w, rec.w + rec.z) >= x1) {      // see stage_culled
                    keep = false;
                    fl ^= row_span_mask(max(rec.x, y0) - y0, min(rec.x + rec.y, y1) - y0);
                }
            }
            const unsigned msk = __ballot_sync(kFull, keep);
            const int pos = cnt + __popc(msk & ((1u << lane) - 1u));
            if (keep && pos < cap) {
                E[pos] = rec;
                R[pos] = rec.y > 0 ? __frcp_rn((float)(2 * rec.y)) : 0.0f;
            }
            cnt += __popc(msk);
        }
    }
    if (right) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fl ^= __shfl_xor_sync(kFull, fl, o);
    }
    flip = fl;
    return cnt;
}

// ----------------------------------------------------------------------------------------------
// a3: candidate pairs (filter). Tiles hold contiguous polygon ranges in both sets.
// ----------------------------------------------------------------------------------------------
__global__ void k_tile_ranges(const int32_t* tile, long long n, int n_tiles, long long* start)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_tiles) return;
    if (!tile) { start[t] = t == 0 ? 0 : n; return; }
    long long lo = 0, hi = n;          // first index with tile[idx] >= t
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if (tile[mid] < t) lo = mid + 1; else hi = mid;
    }
    start[t] = lo;
}

// Per-tile uniform grid over the B polygons. Cell size: about one B polygon per cell (a performance
// choice only; any size gives the same pairs). B polygon b is registered in every cell its closed
// MBR touches; an A polygon probes every cell its closed MBR touches, and a pair (a, b) is reported
// only from the cell holding the corner (max(ax0, bx0), max(ay0, by0)) of the MBR intersection,
// which both MBRs touch: every overlapping pair is found exactly once.
struct TileGrid {
    int ox, oy;        // grid origin (min x0, min y0 of the tile's B MBRs)
    int cell;          // cell size in pixels
    int gx, gy;        // cells per row / column (0 when the tile has no B polygon)
};

__device__ __forceinline__ int floor_div(int n, int d) { return n >= 0 ? n / d : -((-n + d - 1) / d); }

// One warp per tile: bounding box of the tile's B MBRs and the grid laid over it.
__global__ void k_tile_grid(const int4* __restrict__ mbrB, const long long* __restrict__ bstart, int n_tiles,
                            TileGrid* grid, long long* ncells)
{
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
    if (warp >= n_tiles) return;
    const long long b0 = bstart[warp], b1 = bstart[warp + 1];
    int x0 = 0x7fffffff, y0 = 0x7fffffff, x1 = -0x7fffffff, y1 = -0x7fffffff;
    for (long long base = b0; base < b1; base += 32) {
        const long long b = base + lane;
        if (b < b1) {
            const int4 m = mbrB[b];
            x0 = min(x0, m.x); y0 = min(y0, m.y); x1 = max(x1, m.z); y1 = max(y1, m.w);
        }
    }
    x0 = warp_min(x0); y0 = warp_min(y0); x1 = warp_max(x1); y1 = warp_max(y1);
    if (lane != 0) return;
    TileGrid g{0, 0, 1, 0, 0};
    if (b1 > b0) {
        const double area = ((double)(x1 - x0) + 1.0) * ((double)(y1 - y0) + 1.0);
        int cell = (int)ceil(sqrt(area / (double)(b1 - b0)));
        cell = max(cell, 8);
        // at most 4096 cells per axis
        cell = max(cell, (int)(((long long)max(x1 - x0, y1 - y0) + 4095) / 4096));
        g = TileGrid{x0, y0, cell, (x1 - x0) / cell + 1, (y1 - y0) / cell + 1};
    }
    grid[warp] = g;
    ncells[warp] = (long long)g.gx * g.gy;
}

// Sizes of the grid's buffers fixed before the counts are known: ok (when not null) is cleared as
// soon as a count exceeds its buffer, and every kernel after it then does nothing (the caller reads
// ok with the pair count and redoes the call with exact sizes). One thread.
__global__ void k_cap_check(const long long* total, long long cap, unsigned long long* ok, int first)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        const bool fit = *total <= cap;
        *ok = (first ? fit : (*ok != 0ull && fit)) ? 1ull : 0ull;
    }
}

// One thread per B polygon: count its registrations per cell.
__global__ void __launch_bounds__(256) k_bin_count(const int4* __restrict__ mbrB, const int32_t* __restrict__ tileB,
                                                   long long nB, const TileGrid* __restrict__ grid,
                                                   const long long* __restrict__ cellbase,
                                                   unsigned long long* __restrict__ count,
                                                   const unsigned long long* __restrict__ ok)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nB || (ok && !*ok)) return;
    const int t = tileB ? tileB[b] : 0;
    const TileGrid g = grid[t];
    const int4 m = mbrB[b];
    const int cx0 = (m.x - g.ox) / g.cell, cx1 = (m.z - g.ox) / g.cell;
    const int cy0 = (m.y - g.oy) / g.cell, cy1 = (m.w - g.oy) / g.cell;
    const long long base = cellbase[t];
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) atomicAdd(&count[base + (long long)cy * g.gx + cx], 1ull);
}

// One thread per B polygon: place its index in every cell it touches (order within a cell unspecified).
__global__ void __launch_bounds__(256) k_bin_fill(const int4* __restrict__ mbrB, const int32_t* __restrict__ tileB,
                                                  long long nB, const TileGrid* __restrict__ grid,
                                                  const long long* __restrict__ cellbase, int* __restrict__ cursor,
                                                  const long long* __restrict__ cell_off, int* __restrict__ entries,
                                                  const unsigned long long* __restrict__ ok)
{
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nB || (ok && !*ok)) return;
    const int t = tileB ? tileB[b] : 0;
    const TileGrid g = grid[t];
    const int4 m = mbrB[b];
    const int cx0 = (m.x - g.ox) / g.cell, cx1 = (m.z - g.ox) / g.cell;
    const int cy0 = (m.y - g.oy) / g.cell, cy1 = (m.w - g.oy) / g.cell;
    const long long base = cellbase[t];
    for (int cy = cy0; cy <= cy1; ++cy)
        for (int cx = cx0; cx <= cx1; ++cx) {
            const long long c = base + (long long)cy * g.gx + cx;
            entries[cell_off[c] + atomicAdd(&cursor[c], 1)] = (int)b;
        }
}

struct ProbeArgs {
    const int4* mbrA; const int32_t* tileA; long long nA;
    const int4* mbrB;
    const TileGrid* grid; const long long* cellbase; const long long* cell_off; const int* entries;
    int n_tiles;
    const unsigned long long* ok;     // not null: probe nothing unless *ok (see k_cap_check)
};

// The cells an A polygon probes (clamped to its tile's grid); false when there are none.
__device__ __forceinline__ bool probe_range(const ProbeArgs& p, long long a, int4& A, TileGrid& g, long long& base,
                                            int& cx0, int& cx1, int& cy0, int& cy1)
{
    if (p.ok && !*p.ok) return false;
    const int t = p.tileA ? p.tileA[a] : 0;
    if (t >= p.n_tiles) return false;
    g = p.grid[t];
    if (g.gx == 0) return false;
    A = p.mbrA[a];
    cx0 = max(0, floor_div(A.x - g.ox, g.cell)); cx1 = min(g.gx - 1, floor_div(A.z - g.ox, g.cell));
    cy0 = max(0, floor_div(A.y - g.oy, g.cell)); cy1 = min(g.gy - 1, floor_div(A.w - g.oy, g.cell));
    base = p.cellbase[t];
    return cx0 <= cx1 && cy0 <= cy1;
}

// Is b (in cell (cx, cy)) a pair of A reported from this cell?
__device__ __forceinline__ bool pair_here(const int4& A, const int4& B, const TileGrid& g, int cx, int cy)
{
    if (!(A.x <= B.z && B.x <= A.z && A.y <= B.w && B.y <= A.w)) return false;
    const int rx = max(A.x, B.x), ry = max(A.y, B.y);
    return (rx - g.ox) / g.cell == cx && (ry - g.oy) / g.cell == cy;
}

constexpr int kSmallPairs = 32;   // A polygons with at most this many pairs sort them in registers
constexpr int kThreadCells = 8;   // A polygons probing more cells are counted by a warp ...
constexpr int kSerialCells = 64;  // ... and those probing more than this by a whole CTA

// One thread per A polygon: number of pairs, and the B polygons of the first kSmallPairs of them
// (in the order found) in cand[j * nA + a] (j-major: consecutive threads write consecutive words).
// A polygons with more than kSmallPairs pairs, or whose MBR covers more than kSerialCells cells
// (counted afterwards by k_probe_count_big; cand[a] = -1 marks them), are listed for the CTA paths;
// those covering more than kThreadCells cells are listed for k_probe_count_mid (one warp each, so
// that one thread's long walk over many cells does not hold up its warp).
__global__ void __launch_bounds__(256) k_probe_count(const ProbeArgs p, long long* counts, int* big_list,
                                                     unsigned* big_n, int* cand, int* mid_list, unsigned* mid_n)
{
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= p.nA) return;
    int4 A; TileGrid g; long long base; int cx0, cx1, cy0, cy1;
    long long cnt = 0;
    if (probe_range(p, a, A, g, base, cx0, cx1, cy0, cy1)) {
        const long long ncell = (long long)(cx1 - cx0 + 1) * (cy1 - cy0 + 1);
        if (ncell > kSerialCells) {
            counts[a] = 0;
            cand[a] = -1;
            big_list[atomicAdd(big_n, 1u)] = (int)a;
            return;
        }
        if (ncell > kThreadCells) {
            counts[a] = 0;
            mid_list[atomicAdd(mid_n, 1u)] = (int)a;
            return;
        }
        for (int cy = cy0; cy <= cy1; ++cy)
            for (int cx = cx0; cx <= cx1; ++cx) {
                const long long c = base + (long long)cy * g.gx + cx;
                for (long long e = p.cell_off[c]; e < p.cell_off[c + 1]; ++e) {
                    const int b = p.entries[e];
                    if (pair_here(A, p.mbrB[b], g, cx, cy)) {
                        if (cnt < kSmallPairs) cand[cnt * p.nA + a] = b;
                        ++cnt;
                    }
                }
            }
    }
    counts[a] = cnt;
    if (cnt > kSmallPairs) big_list[atomicAdd(big_n, 1u)] = (int)a;
}

// One warp per A polygon listed by k_probe_count for covering kThreadCells + 1 .. kSerialCells cells:
// its pairs counted with the cells spread over the lanes, its first kSmallPairs partners kept in cand
// (lane by lane: a warp prefix sum of the lanes' counts gives each lane its first slot), and, with
// more than kSmallPairs pairs, listed for k_probe_write_big.
__global__ void __launch_bounds__(256) k_probe_count_mid(const ProbeArgs p, const int* __restrict__ mid_list,
                                                         const unsigned* __restrict__ mid_n, long long* counts,
                                                         int* big_list, unsigned* big_n, int* cand)
{
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long nm = *mid_n;
    for (long long j = (long long)blockIdx.x * (blockDim.x >> 5) + warp; j < nm; j += nwarps) {
        const long long a = mid_list[j];
        int4 A; TileGrid g; long long base; int cx0, cx1, cy0, cy1;
        probe_range(p, a, A, g, base, cx0, cx1, cy0, cy1);     // true: listed by k_probe_count
        const int ncx = cx1 - cx0 + 1;
        const int ncell = ncx * (cy1 - cy0 + 1);
        int cnt = 0;
        for (int q = lane; q < ncell; q += 32) {
            const int cx = cx0 + q % ncx, cy = cy0 + q / ncx;
            const long long c = base + (long long)cy * g.gx + cx;
            for (long long e = p.cell_off[c]; e < p.cell_off[c + 1]; ++e)
                cnt += pair_here(A, p.mbrB[p.entries[e]], g, cx, cy);
        }
        int total;
        int k = warp_excl(cnt, lane, total);
        for (int q = lane; q < ncell && k < kSmallPairs; q += 32) {
            const int cx = cx0 + q % ncx, cy = cy0 + q / ncx;
            const long long c = base + (long long)cy * g.gx + cx;
            for (long long e = p.cell_off[c]; e < p.cell_off[c + 1] && k < kSmallPairs; ++e) {
                const int b = p.entries[e];
                if (pair_here(A, p.mbrB[b], g, cx, cy)) cand[(long long)(k++) * p.nA + a] = b;
            }
        }
        if (lane == 0) {
            counts[a] = total;
            if (total > kSmallPairs) big_list[atomicAdd(big_n, 1u)] = (int)a;
        }
    }
}

// One thread per A polygon with 1 to kSmallPairs pairs found by k_probe_count: its B polygons from
// cand, sorted, written at offs[a] (the pairs in ascending (a, b) order).
__global__ void __launch_bounds__(256) k_probe_emit_small(long long nA, const long long* __restrict__ offs,
                                                          const int* __restrict__ cand, int32_t* pa, int32_t* pb,
                                                          long long cap)
{
    const long long a = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (a >= nA) return;
    const long long o = offs[a], n = offs[a + 1] - o;
    if (n == 0 || n > kSmallPairs) return;
    const int b0 = cand[a];
    if (b0 < 0) return;                       // many cells: written by the CTA path
    int buf[kSmallPairs];
    buf[0] = b0;
    for (int k = 1; k < (int)n; ++k) {        // insertion into the sorted prefix
        const int b = cand[k * nA + a];
        int j = k;
        while (j > 0 && buf[j - 1] > b) { buf[j] = buf[j - 1]; --j; }
        buf[j] = b;
    }
    for (int j = 0; j < (int)n; ++j)
        if (o + j < cap) { pa[o + j] = (int32_t)a; pb[o + j] = buf[j]; }
}

// One CTA per listed A polygon that covers more than kSerialCells cells: its pair count, cells
// spread over the threads.
__global__ void __launch_bounds__(256) k_probe_count_big(const ProbeArgs p, const int* __restrict__ big_list,
                                                         const unsigned* __restrict__ big_n, long long* counts)
{
    __shared__ long long wsum[8];
    const unsigned nbig = *big_n;
    for (unsigned bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const long long a = big_list[bi];
        int4 A; TileGrid g; long long base; int cx0, cx1, cy0, cy1;
        if (!probe_range(p, a, A, g, base, cx0, cx1, cy0, cy1)) continue;    // uniform per CTA
        const int ncx = cx1 - cx0 + 1;
        const long long ncell = (long long)ncx * (cy1 - cy0 + 1);
        if (ncell <= kSerialCells) continue;                                  // counted by k_probe_count
        long long cnt = 0;
        for (long long q = threadIdx.x; q < ncell; q += blockDim.x) {
            const int cx = cx0 + (int)(q % ncx), cy = cy0 + (int)(q / ncx);
            const long long c = base + (long long)cy * g.gx + cx;
            for (long long e = p.cell_off[c]; e < p.cell_off[c + 1]; ++e)
                cnt += pair_here(A, p.mbrB[p.entries[e]], g, cx, cy);
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(kFull, cnt, o);
        if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = cnt;
        __syncthreads();
        if (threadIdx.x == 0) {
            long long s = 0;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
            counts[a] = s;
        }
        __syncthreads();
    }
}

// One CTA per listed A polygon (more than kSmallPairs pairs): mark its pairs in a shared bitmap
// over the tile's B range, window by window, and write them in ascending b.
constexpr int kBitmapWords = 2048;    // 65,536 B polygons per window
__global__ void __launch_bounds__(256) k_probe_write_big(const ProbeArgs p, const long long* __restrict__ bstart,
                                                         const long long* __restrict__ offs,
                                                         const int* __restrict__ big_list,
                                                         const unsigned* __restrict__ big_n, int32_t* pa,
                                                         int32_t* pb, long long cap)
{
    __shared__ unsigned bits[kBitmapWords];
    __shared__ int wsum[8];
    __shared__ long long run;
    const unsigned nbig = *big_n;
    for (unsigned bi = blockIdx.x; bi < nbig; bi += gridDim.x) {
        const long long a = big_list[bi];
        int4 A; TileGrid g; long long base; int cx0, cx1, cy0, cy1;
        if (!probe_range(p, a, A, g, base, cx0, cx1, cy0, cy1)) continue;   // uniform per CTA
        const int t = p.tileA ? p.tileA[a] : 0;
        const long long b0 = bstart[t], b1 = bstart[t + 1];
        const int ncx = cx1 - cx0 + 1;
        const long long ncell = (long long)ncx * (cy1 - cy0 + 1);
        if (threadIdx.x == 0) run = offs[a];
        for (long long w0 = b0; w0 < b1; w0 += 32LL * kBitmapWords) {
            for (int i = threadIdx.x; i < kBitmapWords; i += blockDim.x) bits[i] = 0u;
            __syncthreads();
            for (long long q = threadIdx.x; q < ncell; q += blockDim.x) {
                const int cx = cx0 + (int)(q % ncx), cy = cy0 + (int)(q / ncx);
                const long long c = base + (long long)cy * g.gx + cx;
                for (long long e = p.cell_off[c]; e < p.cell_off[c + 1]; ++e) {
                    const int b = p.entries[e];
                    const long long r = (long long)b - w0;
                    if (r >= 0 && r < 32LL * kBitmapWords && pair_here(A, p.mbrB[b], g, cx, cy))
                        atomicOr(&bits[r >> 5], 1u << (r & 31));
                }
            }
            __syncthreads();
            // ordered emission: each thread owns kBitmapWords / blockDim consecutive words
            const int per = kBitmapWords / (int)blockDim.x;
            int mine = 0;
            for (int i = 0; i < per; ++i) mine += __popc(bits[threadIdx.x * per + i]);
            int incl = mine;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int v = __shfl_up_sync(kFull, incl, o);
                if ((threadIdx.x & 31) >= o) incl += v;
            }
            if ((threadIdx.x & 31) == 31) wsum[threadIdx.x >> 5] = incl;
            __syncthreads();
            int before = 0;
            for (int w = 0; w < (int)(threadIdx.x >> 5); ++w) before += wsum[w];
            long long o = run + before + incl - mine;
            for (int i = 0; i < per; ++i) {
                unsigned m = bits[threadIdx.x * per + i];
                while (m) {
                    const int bit = __ffs(m) - 1;
                    m &= m - 1;
                    if (o < cap) { pa[o] = (int32_t)a; pb[o] = (int32_t)(w0 + 32LL * (threadIdx.x * per + i) + bit); }
                    ++o;
                }
            }
            __syncthreads();
            if (threadIdx.x == blockDim.x - 1) run = o;
            __syncthreads();
        }
    }
}

__global__ void k_gather_tile_offsets(const long long* offs, const long long* astart, int n_tiles,
                                      int n_tiles_a, long long nA, int64_t* out)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t > n_tiles) return;
    const long long a = t <= n_tiles_a ? astart[t] : nA;
    out[t] = offs[a];
}

// ----------------------------------------------------------------------------------------------
// device-wide exclusive scan of int64 counts (three passes)
// ----------------------------------------------------------------------------------------------
constexpr int kScanBlock = 1024;

__device__ __forceinline__ long long block_incl_scan(long long v, long long* sh)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long u = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += u;
    }
    if (lane == 31) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        long long s = lane < (int)(blockDim.x >> 5) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const long long u = __shfl_up_sync(kFull, s, o);
            if (lane >= o) s += u;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const long long r = v + (warp > 0 ? sh[warp - 1] : 0);
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_reduce(const long long* in, long long n, long long* bsum)
{
    __shared__ long long sh[32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const long long v = i < n ? in[i] : 0;
    const long long s = block_incl_scan(v, sh);
    if (threadIdx.x == kScanBlock - 1) bsum[blockIdx.x] = s;
}

__global__ void __launch_bounds__(kScanBlock) k_scan_top(long long* bsum, long long nb)
{
    __shared__ long long sh[32];
    __shared__ long long tot;
    long long carry = 0;
    for (long long base = 0; base < nb; base += kScanBlock) {
        const long long i = base + threadIdx.x;
        const long long v = i < nb ? bsum[i] : 0;
        const long long s = block_incl_scan(v, sh);
        if (i < nb) bsum[i] = carry + s - v;   // exclusive
        if (threadIdx.x == kScanBlock - 1) tot = s;
        __syncthreads();
        carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(kScanBlock) k_scan_apply(const long long* in, long long n, const long long* bsum,
                                                           long long* out /* [n+1] */)
{
    __shared__ long long sh[32];
    const long long i = (long long)blockIdx.x * kScanBlock + threadIdx.x;
    const long long v = i < n ? in[i] : 0;
    const long long s = block_incl_scan(v, sh);
    const long long base = bsum[blockIdx.x];
    if (i < n) out[i] = base + s - v;
    if (i == n - 1) out[n] = base + s;
}

// ----------------------------------------------------------------------------------------------
// a4 + a5: pair areas, plain form (one warp per pair, grid-stride)
// ----------------------------------------------------------------------------------------------
struct AreasArgs {
    long long n;
    long long nA, nB;
    const int32_t* pa;
    const int32_t* pb;
    const int64_t* offA; const int32_t* xyA; const int4* mbrA; const int64_t* areaA;
    const int64_t* offB; const int32_t* xyB; const int4* mbrB; const int64_t* areaB;
    int64_t* inter;
    int64_t* uni;
    int T;
    WorkCounters* counters;
    const char* bandsA;     // band index blobs (nullptr = none)
    const char* bandsB;
    int words;              // leaf windows from parity words (1) or as strips against every edge (0)
    // pixel rasters of both sets (all four set, or all null): pair areas from them (raster.cuh)
    const long long* roffA; const uint32_t* rwA;
    const long long* roffB; const uint32_t* rwB;
};

// Block of polygon i in a band index blob (nullptr: no blob, or no block for this polygon).
__device__ __forceinline__ const char* band_block(const char* blob, long long i)
{
    if (!blob) return nullptr;
    const long long at = reinterpret_cast<const long long*>(blob + sizeof(BandHead))[i];
    return at < 0 ? nullptr : blob + at;
}

// Stage both polygons of a pair for the window [x0, x1) x [y0, y1): each keeps only the edges
// that can matter there (from its band block bp / bq when it has one, else from its ring) and is
// resident when those fit the buffer; otherwise it is read chunk by chunk from its whole ring.
template <int CAP, int STK>
__device__ __forceinline__ void stage_pair(PolyPair& pp, const char* bp, int minyp, const char* bq, int minyq,
                                           int x0, int y0, int x1, int y1, WarpSmem<CAP, STK>& S, int lane)
{
    constexpr bool right = CAP > 64;     // see flip_of
    unsigned long long fp = 0, fq = 0;
    const int cp = bp ? stage_banded(bp, minyp, x0, y0, x1, y1, S.ep, S.rp, CAP, lane, right, fp)
                      : stage_culled(pp.vp, pp.np, x0, y0, x1, y1, S.ep, S.rp, CAP, lane, right, fp);
    const int cq = bq ? stage_banded(bq, minyq, x0, y0, x1, y1, S.eq, S.rq, CAP, lane, right, fq)
                      : stage_culled(pp.vq, pp.nq, x0, y0, x1, y1, S.eq, S.rq, CAP, lane, right, fq);
    pp.rp_res = cp <= CAP;
    pp.rq_res = cq <= CAP;
    if (pp.rp_res) pp.np = cp;
    if (pp.rq_res) pp.nq = cq;
    pp.fp = pp.rp_res ? fp : 0;   // a polygon read from its whole ring keeps every edge
    pp.fq = pp.rq_res ? fq : 0;
}

template <int CAP, int STK, bool COUNT>
__global__ void SCCG_ITEM_BOUNDS k_pair_areas_plain(const AreasArgs a)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[warp];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    WorkCounters wc = {};
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp; i < a.n; i += nwarps) {
        const int ia = a.pa[i], ib = a.pb[i];
        int64_t out_i = -1, out_u = -1;      // invalid pair: flagged, not read
        if (ia >= 0 && ia < a.nA && ib >= 0 && ib < a.nB) {
            const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
            const int wx0 = max(ma.x, mb.x), wy0 = max(ma.y, mb.y);
            const int wx1 = min(ma.z, mb.z), wy1 = min(ma.w, mb.w);
            uint32_t inter = 0;
            if (wx1 > wx0 && wy1 > wy0) {
                const long long pa0 = a.offA[ia], pa1 = a.offA[ia + 1];
                const long long qb0 = a.offB[ib], qb1 = a.offB[ib + 1];
                PolyPair pp;
                pp.vp = reinterpret_cast<const int2*>(a.xyA) + pa0; pp.np = (int)(pa1 - pa0);
                pp.vq = reinterpret_cast<const int2*>(a.xyB) + qb0; pp.nq = (int)(qb1 - qb0);
                __syncwarp();
                const char* bp = band_block(a.bandsA, ia);
                const char* bq = band_block(a.bandsB, ib);
                stage_pair(pp, bp, ma.y, bq, mb.y, wx0, wy0, wx1, wy1, S, lane);
                __syncwarp();
                inter = pixelbox<true, COUNT>(pp, wx0, wy0, wx1, wy1, a.T, a.words, S, lane, wc);
            }
            out_i = (int64_t)inter;
            out_u = a.areaA[ia] + a.areaB[ib] - (int64_t)inter;
        }
        if (lane == 0) {
            a.inter[i] = out_i;
            a.uni[i] = out_u;
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// PixelBox-NoSep (Sec. 5.2, Fig. 8): the intersection by PixelBox over MBR(p) n MBR(q) and the union
// counted directly, by the same subdivision over the bounding box of MBR(p) u MBR(q), instead of
// ||p|| + ||q|| - ||p n q||. One warp per pair. Kept for the comparison; requires polygon extents
// of at most kNoSepExtent so that the union window keeps every product in int32.
constexpr int kNoSepExtent = 8192;

template <int CAP, int STK, bool COUNT>
__global__ void SCCG_ITEM_BOUNDS k_pair_areas_nosep(const AreasArgs a)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[warp];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    WorkCounters wc = {};
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + warp; i < a.n; i += nwarps) {
        const int ia = a.pa[i], ib = a.pb[i];
        int64_t out_i = -1, out_u = -1;
        if (ia >= 0 && ia < a.nA && ib >= 0 && ib < a.nB) {
            const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
            const long long pa0 = a.offA[ia], pa1 = a.offA[ia + 1];
            const long long qb0 = a.offB[ib], qb1 = a.offB[ib + 1];
            const char* bp = band_block(a.bandsA, ia);
            const char* bq = band_block(a.bandsB, ib);
            uint32_t cnt[2] = {0, 0};
            for (int u = 0; u < 2; ++u) {
                const int wx0 = u ? min(ma.x, mb.x) : max(ma.x, mb.x), wy0 = u ? min(ma.y, mb.y) : max(ma.y, mb.y);
                const int wx1 = u ? max(ma.z, mb.z) : min(ma.z, mb.z), wy1 = u ? max(ma.w, mb.w) : min(ma.w, mb.w);
                if (wx1 > wx0 && wy1 > wy0) {
                    PolyPair pp;
                    pp.vp = reinterpret_cast<const int2*>(a.xyA) + pa0; pp.np = (int)(pa1 - pa0);
                    pp.vq = reinterpret_cast<const int2*>(a.xyB) + qb0; pp.nq = (int)(qb1 - qb0);
                    __syncwarp();
                    stage_pair(pp, bp, ma.y, bq, mb.y, wx0, wy0, wx1, wy1, S, lane);
                    __syncwarp();
                    cnt[u] = u ? pixelbox<true, COUNT, CAP, STK, true>(pp, wx0, wy0, wx1, wy1, a.T, a.words, S, lane, wc)
                               : pixelbox<true, COUNT>(pp, wx0, wy0, wx1, wy1, a.T, a.words, S, lane, wc);
                }
            }
            out_i = (int64_t)cnt[0];
            out_u = (int64_t)cnt[1];
        }
        if (lane == 0) {
            a.inter[i] = out_i;
            a.uni[i] = out_u;
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// ----------------------------------------------------------------------------------------------
// a7: persistent form. Each pair's window is cut into work items of at most side x side pixels
// (heavy pairs spread over many warps); resident warps pull chunks of items from a device queue.
// ----------------------------------------------------------------------------------------------
__device__ __forceinline__ bool pair_window(const AreasArgs& a, long long i, int& ia, int& ib, int& wx0, int& wy0,
                                            int& wx1, int& wy1)
{
    ia = a.pa[i];
    ib = a.pb[i];
    if (ia < 0 || ia >= a.nA || ib < 0 || ib >= a.nB) return false;
    const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
    wx0 = max(ma.x, mb.x); wy0 = max(ma.y, mb.y);
    wx1 = min(ma.z, mb.z); wy1 = min(ma.w, mb.w);
    return true;
}

// One thread per pair: number of work items; pairs without items get their final values here.
__global__ void k_plan(const AreasArgs a, int side, int cap_small, long long* nitems_s, long long* nitems_b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int ia, ib, wx0, wy0, wx1, wy1;
    long long k = 0;
    bool big = false;
    if (!pair_window(a, i, ia, ib, wx0, wy0, wx1, wy1)) {
        a.inter[i] = -1;
        a.uni[i] = -1;
    } else if (wx1 <= wx0 || wy1 <= wy0) {
        a.inter[i] = 0;
        a.uni[i] = a.areaA[ia] + a.areaB[ib];
    } else {
        k = (long long)((wx1 - wx0 + side - 1) / side) * ((wy1 - wy0 + side - 1) / side);
        if (k > 1) a.inter[i] = 0;     // accumulated by atomics
        big = a.offA[ia + 1] - a.offA[ia] > cap_small || a.offB[ib + 1] - a.offB[ib] > cap_small;
    }
    nitems_s[i] = big ? 0 : k;
    nitems_b[i] = big ? k : 0;
}

// Pairs cut into several items: union from the accumulated intersection.
__global__ void k_union(const AreasArgs a, const long long* nitems_s, const long long* nitems_b)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n || nitems_s[i] + nitems_b[i] <= 1) return;
    a.uni[i] = a.areaA[a.pa[i]] + a.areaB[a.pb[i]] - a.inter[i];
}

// Largest p in [0, n) with ioff[p] <= it (ioff non-decreasing, ioff[0] = 0, it < ioff[n]):
// 32-ary search, one probe per lane per round. Whole warp, converged.
__device__ __forceinline__ long long find_pair(const long long* ioff, long long n, long long it, int lane)
{
    long long lo = 0, hi = n;   // ioff[lo] <= it, and the answer is < hi
    while (hi - lo > 1) {
        const long long step = (hi - lo + 31) / 32;
        const long long pos = lo + (long long)lane * step;
        const bool ok = pos < hi && ioff[pos] <= it;
        const unsigned m = __ballot_sync(kFull, ok);
        const int L = 31 - __clz(m);          // lane 0 always qualifies (ioff[lo] <= it)
        lo = lo + (long long)L * step;
        hi = min(lo + step, hi);
    }
    return lo;
}

#ifndef SCCG_ITEM_CHUNK
#define SCCG_ITEM_CHUNK 4
#endif
#ifndef SCCG_ITEM_CHUNK_MAX
#define SCCG_ITEM_CHUNK_MAX 64
#endif
// Items a warp takes from a queue at a time: guided self-scheduling, a quarter of the remaining
// items' share per warp, between these bounds (large takes early spread the pair search over many
// items, small ones at the end keep the tail short).
constexpr int kItemChunk = SCCG_ITEM_CHUNK;
constexpr int kItemChunkMax = SCCG_ITEM_CHUNK_MAX;

// Overflow list entries: pair index and sub-window, packed (no search needed to find the pair).
__device__ __forceinline__ unsigned long long ovf_pack(long long i, long long sub)
{
    return ((unsigned long long)i << 32) | (unsigned long long)(uint32_t)sub;
}

// One work item: sub-window `sub` of pair i's window, cut into side x side items. With OVF, an item
// whose window-culled edges do not fit the buffers is appended to the overflow list (for a kernel
// with larger buffers) instead of being read chunk by chunk from the whole rings; when the list is
// full the item is done here anyway. Whole warp, converged.
template <int CAP, int STK, bool COUNT, bool OVF>
__device__ __forceinline__ void do_item(const AreasArgs a, int side, const long long* nitems, long long i,
                                        long long sub, unsigned long long* ovf_list, unsigned long long* ovf_n,
                                        long long ovf_cap, WarpSmem<CAP, STK>& S, int lane, WorkCounters& wc)
{
    const int ia = a.pa[i], ib = a.pb[i];
    const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
    const int wx0 = max(ma.x, mb.x), wy0 = max(ma.y, mb.y);
    const int wx1 = min(ma.z, mb.z), wy1 = min(ma.w, mb.w);
    const int gx = (wx1 - wx0 + side - 1) / side;
    const int sx = (int)(sub % gx), sy = (int)(sub / gx);
    const int x0 = wx0 + sx * side, y0 = wy0 + sy * side;
    const int x1 = min(x0 + side, wx1), y1 = min(y0 + side, wy1);
    const long long pa0 = a.offA[ia], pa1 = a.offA[ia + 1];
    const long long qb0 = a.offB[ib], qb1 = a.offB[ib + 1];
    PolyPair pp;
    pp.vp = reinterpret_cast<const int2*>(a.xyA) + pa0; pp.np = (int)(pa1 - pa0);
    pp.vq = reinterpret_cast<const int2*>(a.xyB) + qb0; pp.nq = (int)(qb1 - qb0);
    __syncwarp();
    stage_pair(pp, band_block(a.bandsA, ia), ma.y, band_block(a.bandsB, ib), mb.y, x0, y0, x1, y1, S, lane);
    __syncwarp();
    if (OVF && !(pp.rp_res && pp.rq_res)) {
        unsigned long long slot = 0;
        if (lane == 0) slot = atomicAdd(ovf_n, 1ull);
        slot = __shfl_sync(kFull, slot, 0);
        if ((long long)slot < ovf_cap) {
            if (lane == 0) ovf_list[slot] = ovf_pack(i, sub);
            return;
        }
    }
    const uint32_t cnt = pixelbox<true, COUNT>(pp, x0, y0, x1, y1, a.T, a.words, S, lane, wc);
    if (lane == 0) {
        if (nitems[i] == 1) {
            a.inter[i] = (int64_t)cnt;
            a.uni[i] = a.areaA[ia] + a.areaB[ib] - (int64_t)cnt;
        } else {
            atomicAdd(reinterpret_cast<unsigned long long*>(a.inter + i), (unsigned long long)cnt);
        }
    }
}

// Persistent pair areas over one item queue (items of pair i: ioff[i] .. ioff[i+1]-1): resident
// warps take kItemChunk items at a time from the queue head.
template <int CAP, int STK, bool COUNT, bool OVF>
__global__ void SCCG_ITEM_BOUNDS k_pair_areas_persistent(const AreasArgs a, int side, const long long* nitems,
                                                               const long long* ioff, unsigned long long* head,
                                                               unsigned long long* ovf_list, unsigned long long* ovf_n,
                                                               long long ovf_cap)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[warp];
    WorkCounters wc = {};
    const long long total = ioff[a.n];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long seen = 0;                        // queue head at this warp's last take (<= the current one)
    for (;;) {
        const long long take = min((long long)kItemChunkMax, max((long long)kItemChunk, (total - seen) / (4 * nwarps)));
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(head, (unsigned long long)take);
        first = __shfl_sync(kFull, first, 0);
        if ((long long)first >= total) break;
        seen = (long long)first;
        const long long last = min((long long)first + take, total);
        long long i = find_pair(ioff, a.n, (long long)first, lane);
        for (long long it = (long long)first; it < last; ++it) {
            if (ioff[i + 1] <= it) {                  // warp-uniform: next pair, else search again
                ++i;
                if (ioff[i + 1] <= it) i = find_pair(ioff, a.n, it, lane);
            }
            do_item<CAP, STK, COUNT, OVF>(a, side, nitems, i, it - ioff[i], ovf_list, ovf_n, ovf_cap, S, lane, wc);
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// The items another launch appended to its overflow list, one at a time from a second queue head.
// With OVF, items that do not fit these buffers either are appended in turn to list 2 (for a launch
// with larger buffers).
template <int CAP, int STK, bool COUNT, bool OVF>
__global__ void SCCG_ITEM_BOUNDS k_pair_areas_overflow(const AreasArgs a, int side, const long long* nitems,
                                                             const unsigned long long* ovf_list,
                                                             const unsigned long long* ovf_n, long long ovf_cap,
                                                             unsigned long long* head, unsigned long long* ovf2_list,
                                                             unsigned long long* ovf2_n, long long ovf2_cap)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WarpSmem<CAP, STK>& S = reinterpret_cast<WarpSmem<CAP, STK>*>(smem4)[warp];
    WorkCounters wc = {};
    const long long n = min((long long)*ovf_n, ovf_cap);
    for (;;) {
        unsigned long long j = 0;
        if (lane == 0) j = atomicAdd(head, 1ull);
        j = __shfl_sync(kFull, j, 0);
        if ((long long)j >= n) break;
        const unsigned long long e = ovf_list[j];
        do_item<CAP, STK, COUNT, OVF>(a, side, nitems, (long long)(e >> 32), (long long)(uint32_t)e, ovf2_list, ovf2_n,
                                      ovf2_cap, S, lane, wc);
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// Small transfers done by kernels instead of the copy engines, so that they are never queued behind
// a bulk host-to-device copy of the next batch (pinned host memory is addressed directly).
__global__ void k_copy64(const unsigned long long* src, unsigned long long* dst, int n)
{
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
}

// Bulk copy by the SMs (sccg_copy): n units of T with a grid stride, four loads in flight per
// thread; the tail_words 4-byte words after the units by the first threads of block 0. Either
// side may be page-locked host memory addressed directly over the host link.
template <class T>
__global__ void __launch_bounds__(512) k_copy_units(const T* __restrict__ src, T* __restrict__ dst, long long n,
                                                    const uint32_t* __restrict__ src_tail, uint32_t* __restrict__ dst_tail,
                                                    int tail_words)
{
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    const long long step = (long long)gridDim.x * blockDim.x;
    for (; i + 3 * step < n; i += 4 * step) {
        const T u0 = src[i], u1 = src[i + step], u2 = src[i + 2 * step], u3 = src[i + 3 * step];
        dst[i] = u0;
        dst[i + step] = u1;
        dst[i + 2 * step] = u2;
        dst[i + 3 * step] = u3;
    }
    for (; i < n; i += step) dst[i] = src[i];
    if (blockIdx.x == 0 && (int)threadIdx.x < tail_words) dst_tail[threadIdx.x] = src_tail[threadIdx.x];
}

__global__ void k_zero32(uint32_t* p, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        p[i] = 0u;
}

// ----------------------------------------------------------------------------------------------
// Streaming form of the persistent pair areas, for items that are one leaf each (side^2 < T, parity
// words): the leaf's parity words are XORed straight from the polygons' rings (or their band
// blocks), 32 edges at a time held in registers, so no edge buffer bounds a polygon's size, the
// shared memory per warp is the two polygons' parity words only, and every item goes to one queue.
// ----------------------------------------------------------------------------------------------
struct StreamSmem {
    XorRows xp;
    XorRows xq;
};


// ... of the edge records listed in the band block `blk` (polygon minimum y `miny`) for the bands
// of those rows; a record listed in several of them is taken from the first (as stage_banded).
__device__ __forceinline__ void xor_stream_bands(const char* blk, int miny, int x0, int y0, int nr, int W, int nw,
                                                 XorRows& X, int lane, unsigned long long& entries)
{
    const int* head = reinterpret_cast<const int*>(blk);
    const int nb = head[0];
    const int* boff = head + 4;
    const int4* ent = reinterpret_cast<const int4*>(blk + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
    const int b0 = min(max((y0 - miny) >> kBandShift, 0), nb - 1);
    const int b1 = min(max((y0 + nr - 1 - miny) >> kBandShift, 0), nb - 1);
    for (int b = b0; b <= b1; ++b) {
        const int e0 = boff[b], e1 = boff[b + 1];
        for (int base = e0; base < e1; base += 32) {
            const int k = base + lane;
            bool has = false;
            int4 rec = make_int4(0, 0, 0, 0);
            if (k < e1) {
                rec = ent[k];
                has = max(b0, (rec.x - miny) >> kBandShift) == b;
            }
            xor_group(has, rec.x, rec.y, rec.z, rec.w, x0, y0, nr, W, nw, X, lane, entries);
        }
    }
}


// Work item `sub` of pair i (as do_item), one leaf, streamed. Whole warp, converged.
template <bool COUNT>
__device__ __forceinline__ void do_item_stream(const AreasArgs a, int side, const long long* nitems, long long i,
                                               long long sub, StreamSmem& S, int lane, WorkCounters& wc)
{
    const int ia = a.pa[i], ib = a.pb[i];
    const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
    const int wx0 = max(ma.x, mb.x), wy0 = max(ma.y, mb.y);
    const int wx1 = min(ma.z, mb.z), wy1 = min(ma.w, mb.w);
    const int gx = (wx1 - wx0 + side - 1) / side;
    const int sx = (int)(sub % gx), sy = (int)(sub / gx);
    const int x0 = wx0 + sx * side, y0 = wy0 + sy * side;
    const int x1 = min(x0 + side, wx1), y1 = min(y0 + side, wy1);
    const int W = x1 - x0, H = y1 - y0;
    const int2* vp = reinterpret_cast<const int2*>(a.xyA) + a.offA[ia];
    const int np = (int)(a.offA[ia + 1] - a.offA[ia]);
    const int2* vq = reinterpret_cast<const int2*>(a.xyB) + a.offB[ib];
    const int nq = (int)(a.offB[ib + 1] - a.offB[ib]);
    const char* bp = band_block(a.bandsA, ia);
    const char* bq = band_block(a.bandsB, ib);
    if (COUNT && lane == 0) wc.window_pixels += (unsigned long long)W * H;
    uint32_t acc = 0;
    for (int cx = 0; cx < W; cx += 32 * kXorMaxWords) {
        const int Wp = min(32 * kXorMaxWords, W - cx), nw = (Wp + 31) >> 5;
        const int nr = min(64, kXorWords / nw);
        for (int r0 = 0; r0 < H; r0 += nr) {
            const int nrr = min(nr, H - r0);
            __syncwarp();
            for (int k = lane; k < nrr; k += 32) {
                S.xp.F[k] = 0;
                S.xq.F[k] = 0;
            }
            for (int k = lane; k < nrr * nw; k += 32) {
                S.xp.P[k] = 0;
                S.xq.P[k] = 0;
            }
            __syncwarp();
            unsigned long long ce = 0;
            if (bp) xor_stream_bands(bp, ma.y, x0 + cx, y0 + r0, nrr, Wp, nw, S.xp, lane, ce);
            else xor_stream_ring(vp, np, x0 + cx, y0 + r0, nrr, Wp, nw, S.xp, lane, ce);
            if (bq) xor_stream_bands(bq, mb.y, x0 + cx, y0 + r0, nrr, Wp, nw, S.xq, lane, ce);
            else xor_stream_ring(vq, nq, x0 + cx, y0 + r0, nrr, Wp, nw, S.xq, lane, ce);
            __syncwarp();
            for (int k = lane; k < nrr; k += 32) {
                for (int j = 0; j < nw; ++j) {
                    const uint32_t in = __funnelshift_lc(0xffffffffu, 0u, (unsigned)min(32, Wp - 32 * j));
                    acc += __popc(in & xor_word(S.xp, k, nw, j) & xor_word(S.xq, k, nw, j));
                }
                if (COUNT) {
                    wc.row_edges += (unsigned long long)nw;
                    wc.leaf_pixels += (unsigned long long)Wp * 2;
                }
            }
            if (COUNT) wc.row_entries += ce;
        }
    }
    const uint32_t cnt = warp_sum(acc);
    if (lane == 0) {
        if (nitems[i] == 1) {
            a.inter[i] = (int64_t)cnt;
            a.uni[i] = a.areaA[ia] + a.areaB[ib] - (int64_t)cnt;
        } else {
            atomicAdd(reinterpret_cast<unsigned long long*>(a.inter + i), (unsigned long long)cnt);
        }
    }
}

// Persistent streaming pair areas over one item queue (guided self-scheduling, as
// k_pair_areas_persistent).
template <bool COUNT>
__global__ void __launch_bounds__(256, SCCG_STREAM_MIN_BLOCKS) k_pair_areas_stream(const AreasArgs a, int side, const long long* nitems,
                                                     const long long* ioff, unsigned long long* head)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    StreamSmem& S = reinterpret_cast<StreamSmem*>(smem4)[warp];
    WorkCounters wc = {};
    const long long total = ioff[a.n];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long seen = 0;
    for (;;) {
        const long long take = min((long long)kItemChunkMax, max((long long)kItemChunk, (total - seen) / (4 * nwarps)));
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(head, (unsigned long long)take);
        first = __shfl_sync(kFull, first, 0);
        if ((long long)first >= total) break;
        seen = (long long)first;
        const long long last = min((long long)first + take, total);
        long long i = find_pair(ioff, a.n, (long long)first, lane);
        for (long long it = (long long)first; it < last; ++it) {
            if (ioff[i + 1] <= it) {
                ++i;
                if (ioff[i + 1] <= it) i = find_pair(ioff, a.n, it, lane);
            }
            do_item_stream<COUNT>(a, side, nitems, i, it - ioff[i], S, lane, wc);
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// ----------------------------------------------------------------------------------------------
// Leaf form of the persistent pair areas, for items of at most 64 x 64 pixels that are one leaf each
// (side <= 64, side^2 < T): both polygons' parity rows are XORed from their rings (or band blocks)
// streamed as one edge sequence (leaf64.cuh). Each warp reads the data of 32 consecutive pairs at
// once into a shared table (one lane per pair: item range, MBRs, ring pointers and sizes, band blocks,
// ||p|| + ||q||), so the dependent index -> MBR -> offset loads are paid once per 32 pairs instead of
// at the start of every item.
// ----------------------------------------------------------------------------------------------
struct LeafPair {
    long long i0, i1;           // the pair's items: i0 .. i1 - 1
    int4 ma, mb;                // MBRs of p and q
    const int2* vp;
    const int2* vq;
    const char* bp;             // band blocks (nullptr: none)
    const char* bq;
    long long sum_area;         // ||p|| + ||q||
    int np, nq;
};

struct LeafSmem {
    Leaf64 L;
    LeafPair tab[32];
};
static_assert(sizeof(Leaf64) % 16 == 0 && sizeof(LeafPair) % 16 == 0, "LeafSmem keeps its int4 fields aligned");

// ... of the edge records listed in band block `blk` (polygon minimum y `miny`) for the bands of rows
// y0 .. y0 + H - 1, into the rows at word `base`; a record listed in several of those bands is taken
// from the first (as xor_stream_bands). Whole warp, converged.
template <bool COUNT>
__device__ __forceinline__ void leaf_bands(const char* blk, int miny, int base, int x0, int y0, int W, int H,
                                           Leaf64& L, int lane, unsigned long long& entries)
{
    const int* head = reinterpret_cast<const int*>(blk);
    const int nb = head[0];
    const int* boff = head + 4;
    const int4* ent = reinterpret_cast<const int4*>(blk + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
    const int b0 = min(max((y0 - miny) >> kBandShift, 0), nb - 1);
    const int b1 = min(max((y0 + H - 1 - miny) >> kBandShift, 0), nb - 1);
    for (int b = b0; b <= b1; ++b) {
        const int e0 = boff[b], e1 = boff[b + 1];
        for (int k0 = e0; k0 < e1; k0 += 32) {
            const int k = k0 + lane;
            bool has = false;
            int4 rec = make_int4(0, 0, 0, 0);
            if (k < e1) {
                rec = ent[k];
                has = max(b0, (rec.x - miny) >> kBandShift) == b;
            }
            // record {ylo, dy, dx, xl}: lower endpoint (xl, ylo), upper (xl + dx, ylo + dy)
            leaf_batch<COUNT>(has, make_int2(rec.w, rec.x), make_int2(rec.w + rec.z, rec.x + rec.y), x0, y0, W, H,
                              base, L, lane, entries);
        }
    }
}

// Lane j: the table entry of pair i + j. Whole warp.
__device__ __forceinline__ void leaf_fill(const AreasArgs& a, const long long* ioff, long long i, LeafPair* tab,
                                          int lane)
{
    const long long p = i + lane;
    LeafPair e;
    e.i0 = e.i1 = 0x7fffffffffffffffLL;
    e.ma = e.mb = make_int4(0, 0, 0, 0);
    e.vp = e.vq = nullptr;
    e.bp = e.bq = nullptr;
    e.sum_area = 0;
    e.np = e.nq = 0;
    if (p < a.n) {
        e.i0 = ioff[p];
        e.i1 = ioff[p + 1];
        if (e.i1 > e.i0) {               // a pair with items has valid indices (k_plan)
            const int ia = a.pa[p], ib = a.pb[p];
            e.ma = a.mbrA[ia];
            e.mb = a.mbrB[ib];
            const long long oa = a.offA[ia], ob = a.offB[ib];
            e.np = (int)(a.offA[ia + 1] - oa);
            e.nq = (int)(a.offB[ib + 1] - ob);
            e.vp = reinterpret_cast<const int2*>(a.xyA) + oa;
            e.vq = reinterpret_cast<const int2*>(a.xyB) + ob;
            e.bp = band_block(a.bandsA, ia);
            e.bq = band_block(a.bandsB, ib);
            e.sum_area = a.areaA[ia] + a.areaB[ib];
        }
    }
    tab[lane] = e;
}

// Item `sub` of pair pi (table entry te), one leaf of at most 64 x 64 pixels, its rings (or band
// blocks) streamed from global memory. Whole warp, converged.
template <bool COUNT>
__device__ __forceinline__ void leaf_item(const AreasArgs& a, int side, const LeafPair& te, long long pi,
                                          long long sub, Leaf64& L, int lane, WorkCounters& wc)
{
    const int4 ma = te.ma, mb = te.mb;
    const int wx0 = max(ma.x, mb.x), wy0 = max(ma.y, mb.y);
    const int wx1 = min(ma.z, mb.z), wy1 = min(ma.w, mb.w);
    const bool single = te.i1 - te.i0 == 1;
    int x0 = wx0, y0 = wy0;
    if (!single) {        // sub-window sub of gx per row (fewer than 2^31 items per pair)
        const int gx = (wx1 - wx0 + side - 1) / side;
        const int sy = (int)sub / gx;
        x0 += ((int)sub - sy * gx) * side;
        y0 += sy * side;
    }
    const int W = min(x0 + side, wx1) - x0, H = min(y0 + side, wy1) - y0;
    if (W <= 0 || H <= 0 || W > kLeafSide || H > kLeafSide) return;     // not an item of this kernel
    const int2* vp = te.vp;
    const int2* vq = te.vq;
    const char* bp = te.bp;
    const char* bq = te.bq;
    const int np = te.np, nq = te.nq;
    const long long sum_area = te.sum_area;
    if (COUNT && lane == 0) wc.window_pixels += (unsigned long long)W * H;
    __syncwarp();
    leaf_clear(L, W, H, true, lane);
    __syncwarp();
    unsigned long long ce = 0;
    if (!bp && !bq) {
        leaf_rings<COUNT>(vp, np, 0, vq, nq, kLeafQ, x0, y0, W, H, L, lane, ce);
    } else {
        if (bp) leaf_bands<COUNT>(bp, ma.y, 0, x0, y0, W, H, L, lane, ce);
        else leaf_rings<COUNT>(vp, np, 0, vp, 0, 0, x0, y0, W, H, L, lane, ce);
        if (bq) leaf_bands<COUNT>(bq, mb.y, kLeafQ, x0, y0, W, H, L, lane, ce);
        else leaf_rings<COUNT>(vq, nq, kLeafQ, vq, 0, kLeafQ, x0, y0, W, H, L, lane, ce);
    }
    __syncwarp();
    const uint32_t cnt = leaf_pixels<COUNT>(L, W, H, true, lane, wc);
    if (COUNT) wc.row_entries += ce;
    if (lane == 0) {
        if (single) {
            a.inter[pi] = (int64_t)cnt;
            a.uni[pi] = sum_area - (int64_t)cnt;
        } else {
            atomicAdd(reinterpret_cast<unsigned long long*>(a.inter + pi), (unsigned long long)cnt);
        }
    }
}

// Persistent leaf pair areas over one item queue (guided self-scheduling, as k_pair_areas_stream).
template <bool COUNT>
__global__ void __launch_bounds__(256, SCCG_LEAF_MIN_BLOCKS) k_pair_areas_leaf(const AreasArgs a, int side,
                                                                               const long long* ioff,
                                                                               unsigned long long* head)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    LeafSmem& S = reinterpret_cast<LeafSmem*>(smem4)[warp];
    WorkCounters wc = {};
    const long long total = ioff[a.n];
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    long long seen = 0;
    for (;;) {
        const long long take = min((long long)kItemChunkMax, max((long long)kItemChunk, (total - seen) / (4 * nwarps)));
        unsigned long long first = 0;
        if (lane == 0) first = atomicAdd(head, (unsigned long long)take);
        first = __shfl_sync(kFull, first, 0);
        if ((long long)first >= total) break;
        seen = (long long)first;
        const long long last = min((long long)first + take, total);
        long long i = find_pair(ioff, a.n, (long long)first, lane);
        long long it = (long long)first;
        while (it < last) {
            __syncwarp();
            leaf_fill(a, ioff, i, S.tab, lane);
            __syncwarp();
            int j = 0;
            while (it < last) {
                while (j < 32 && S.tab[j].i1 <= it) ++j;      // warp-uniform (shared table)
                if (j == 32) break;
                leaf_item<COUNT>(a, side, S.tab[j], i + j, it - S.tab[j].i0, S.L, lane, wc);
                ++it;
            }
            i += 32;
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// ----------------------------------------------------------------------------------------------
// One lane per pair (threads per pair = 1) for pairs whose window is at most 32 x 32 pixels and
// whose rings are short: the lane streams both rings itself and keeps the two polygons' parity rows
// in its own column of the warp's shared memory (word (row << 5) | lane: every lane in its own bank,
// no atomics), so the warp-wide steps of the leaf kernel (batch setup, span maxima, prefix sums,
// owner searches, reductions) disappear and 32 pairs progress at once.
// ----------------------------------------------------------------------------------------------
constexpr int kLaneSide = 32;            // largest window side of a lane pair
#ifndef SCCG_LANE_MAX_EDGES
#define SCCG_LANE_MAX_EDGES 64
#endif
constexpr int kLaneMaxEdges = SCCG_LANE_MAX_EDGES;   // edges of both rings of a lane pair, at most

struct LaneSmem {
    uint32_t r[2 * kLaneSide][32];       // [row][lane]: rows 0..31 of P, then of Q
    int2 v[kLaneMaxEdges][32];           // [vertex][lane]: the lane's P ring, then its Q ring
};

// Asynchronous 8-byte global -> shared copy (cp.async), and waiting for all of this thread's.
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// k_plan for the leaf kernel. With `lanes`, pairs with a window of at most kLaneSide x kLaneSide
// pixels and at most kLaneMaxEdges edges in both rings get lane[i] = 1 and no items (the lane kernel
// does them whole); the others get their items as in k_plan (lane[i] = 0).
__global__ void k_plan_leaf(const AreasArgs a, int side, int lanes, long long* nitems, long long* lane)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= a.n) return;
    int ia, ib, wx0, wy0, wx1, wy1;
    long long k = 0;
    bool by_lane = false;
    if (!pair_window(a, i, ia, ib, wx0, wy0, wx1, wy1)) {
        a.inter[i] = -1;
        a.uni[i] = -1;
    } else if (wx1 <= wx0 || wy1 <= wy0) {
        a.inter[i] = 0;
        a.uni[i] = a.areaA[ia] + a.areaB[ib];
    } else {
        const long long e = (a.offA[ia + 1] - a.offA[ia]) + (a.offB[ib + 1] - a.offB[ib]);
        by_lane = lanes && wx1 - wx0 <= kLaneSide && wy1 - wy0 <= kLaneSide && e <= kLaneMaxEdges;
        if (!by_lane) {
            k = (long long)((wx1 - wx0 + side - 1) / side) * ((wy1 - wy0 + side - 1) / side);
            if (k > 1) a.inter[i] = 0;     // accumulated by atomics
        }
    }
    nitems[i] = k;
    lane[i] = by_lane ? 1 : 0;
}

// The parity rows of ring vp[0 .. np) (rows 0 .. H-1 of the lane's column) and, when nq > 0, of ring
// vq[0 .. nq) (rows kLaneSide ..) over the window [x0, x0 + W) x [y0, y0 + H), W, H <= kLaneSide.
// The rings are walked as one edge sequence; each step either takes the next edge (its rows
// straddled inside the window, set up as leaf_batch does) or XORs the crossing of the current edge
// with its next row into the row's word (leaf_cross's rule: the first c = ceil(N / 2dy) pixels right
// of x0 flip), so the lane's trip count is its edges plus its crossings. R: the lane's column,
// R[row << 5]. Returns the number of (edge, row) crossings.
template <int STRIDE>
__device__ __forceinline__ unsigned lane_walk(const int2* vp, int np, const int2* vq, int nq, int x0, int y0, int H,
                                              uint32_t* R)
{
    for (int r = 0; r < H; ++r) {
        R[r << 5] = 0u;
        if (nq) R[(kLaneSide + r) << 5] = 0u;
    }
    const int2* v = vp;
    int n = np, j = 1, rowbase = 0;
    int2 prev = vp[(np - 1) * STRIDE];
    int2 nxt = vp[0];
    int s = 0, span = 0, N = 0, dx2 = 0, cap = 0, w = 0;
    float rc = 1.0f;
    unsigned crossings = 0;
    for (;;) {
        if (s >= span) {
            if (j > n) {                        // this ring is done
                if (rowbase || nq == 0) break;
                v = vq;
                n = nq;
                j = 1;
                rowbase = kLaneSide;
                prev = vq[(nq - 1) * STRIDE];
                nxt = vq[0];
            }
            const int2 cur = nxt;
            if (j < n) nxt = v[j * STRIDE];     // the next edge's vertex, loaded ahead
            ++j;
            const bool up = prev.y <= cur.y;
            const int ylo = up ? prev.y : cur.y, yhi = up ? cur.y : prev.y;
            const int xl = up ? prev.x : cur.x, xh = up ? cur.x : prev.x;
            const int rlo = max(ylo, y0);
            span = max(prev.x, cur.x) > x0 ? max(min(yhi, y0 + H) - rlo, 0) : 0;
            s = 0;
            if (span > 0) {
                const int dy = yhi - ylo, dx = xh - xl;
                dx2 = dx + dx;
                N = (2 * (rlo - ylo) + 1) * dx - (2 * (x0 - xl) + 1) * dy;
                cap = (dy + dy) << 5;
                rc = rcp_approx(small_int_to_float(dy + dy));
                w = rowbase + rlo - y0;
                crossings += (unsigned)span;
            }
            prev = cur;
        }
        if (s < span) {
            const int c = leaf_ceil_div(min(max(N, 0), cap), rc);
            R[(w + s) << 5] ^= low_mask(c);
            N += dx2;
            ++s;
        }
    }
    return crossings;
}

// ||p n q|| of a lane pair (lane_walk over both rings staged in the lane's column, then the rows
// inside both, W columns).
constexpr int kLaneStride = 32;          // int2 steps between a lane's consecutive staged vertices
template <bool COUNT>
__device__ __forceinline__ uint32_t lane_pair_inter(const int2* vp, int np, const int2* vq, int nq, int x0, int y0,
                                                    int W, int H, uint32_t* R, WorkCounters& wc)
{
    const unsigned crossings = lane_walk<kLaneStride>(vp, np, vq, nq, x0, y0, H, R);
    const uint32_t vm = low_mask(W);
    uint32_t acc = 0;
    for (int r = 0; r < H; ++r) acc += __popc(R[r << 5] & R[(kLaneSide + r) << 5] & vm);
    if (COUNT) {
        wc.row_entries += crossings;
        wc.row_edges += (unsigned long long)H;
        wc.leaf_pixels += 2ull * W * H;
        wc.window_pixels += (unsigned long long)W * H;
    }
    return acc;
}

// Every pair k_plan_leaf marked (lane[i] = 1), one per lane: each warp takes 32 consecutive pairs,
// every lane copies its pair's two rings into its column of shared memory with asynchronous copies
// (all in flight at once; vertex k of the lane at v[k][lane], so the lanes' later reads of their own
// k-th vertices fall in different banks), then walks them. Grid-stride over groups of 32 pairs.
template <bool COUNT>
__global__ void __launch_bounds__(64, SCCG_LANE_MIN_BLOCKS) k_pair_areas_lanes(const AreasArgs a,
                                                                               const long long* lane)
{
    SCCG_DYNAMIC_SMEM(int4, smem4);
    const int warp = threadIdx.x >> 5, ln = threadIdx.x & 31;
    LaneSmem& S = reinterpret_cast<LaneSmem*>(smem4)[warp];
    uint32_t* R = &S.r[0][ln];
    WorkCounters wc = {};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < a.n; base += stride) {
        const long long p = base + ln;
        bool mine = p < a.n && lane[p] == 1;
        int ia = 0, ib = 0, x0 = 0, y0 = 0, W = 0, H = 0, np = 0, nq = 0;
        const int2* vp = nullptr;
        const int2* vq = nullptr;
        if (mine) {
            ia = a.pa[p];
            ib = a.pb[p];
            const int4 ma = a.mbrA[ia], mb = a.mbrB[ib];
            x0 = max(ma.x, mb.x);
            y0 = max(ma.y, mb.y);
            W = min(ma.z, mb.z) - x0;
            H = min(ma.w, mb.w) - y0;
            const long long oa = a.offA[ia], ob = a.offB[ib];
            np = (int)(a.offA[ia + 1] - oa);
            nq = (int)(a.offB[ib + 1] - ob);
            vp = reinterpret_cast<const int2*>(a.xyA) + oa;
            vq = reinterpret_cast<const int2*>(a.xyB) + ob;
            mine = W > 0 && H > 0 && W <= kLaneSide && H <= kLaneSide && np + nq <= kLaneMaxEdges;
        }
        __syncwarp();                                  // the lanes are done with the previous columns
        if (mine) {
            for (int k = 0; k < np; ++k) cp_async8(&S.v[k][ln], vp + k);
            for (int k = 0; k < nq; ++k) cp_async8(&S.v[np + k][ln], vq + k);
        }
        cp_async_wait_all();
        if (mine) {
            const uint32_t cnt = lane_pair_inter<COUNT>(&S.v[0][ln], np, &S.v[np][ln], nq, x0, y0, W, H, R, wc);
            a.inter[p] = (int64_t)cnt;
            a.uni[p] = a.areaA[ia] + a.areaB[ib] - (int64_t)cnt;
        }
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// Chunk-local candidate pairs to indices into the whole sets (pipelined front end).
__global__ void k_rebase_pairs(int32_t* pa, int32_t* pb, long long n, int base_a, int base_b)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
        pa[i] += base_a;
        pb[i] += base_b;
    }
}

// ----------------------------------------------------------------------------------------------
// Other operators through the same results (Sec. 3.4, implications of PixelBox for other spatial
// operators): ST_Contains from the areas, ST_Touches from edge and vertex tests.
// ----------------------------------------------------------------------------------------------
// bit 0: the A polygon contains the B polygon (||p n q|| = ||q|| > 0); bit 1: the B polygon contains
// the A polygon (||p n q|| = ||p|| > 0); 0xff for a pair whose indices or intersection are invalid.
__global__ void k_contains(const int32_t* pa, const int32_t* pb, const int64_t* inter, const int64_t* areaA,
                           const int64_t* areaB, long long nA, long long nB, long long n, uint8_t* out)
{
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const int ia = pa[k], ib = pb[k];
        if (ia < 0 || ia >= nA || ib < 0 || ib >= nB || inter[k] < 0) { out[k] = 0xff; continue; }
        const int64_t ap = areaA[ia], aq = areaB[ib], x = inter[k];
        out[k] = (uint8_t)(((x == aq && aq > 0) ? 1 : 0) | ((x == ap && ap > 0) ? 2 : 0));
    }
}

__device__ __forceinline__ int orient_sign64(long long ax, long long ay, long long bx, long long by, long long cx,
                                             long long cy)
{
    const long long v = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    return (v > 0) - (v < 0);
}

// One polygon's vertices (lane k: vertex base + k) against the other polygon's edges: whether an
// edge of `w` crosses the edge starting at the lane's vertex properly, whether the vertex lies on an
// edge of `w`, and its even-odd parity against `w` (half-open y-ranges). Whole warp (uniform nw).
__device__ __forceinline__ void vertex_vs_ring(const int2* u, int nu, int k, const int2* w, int nw, bool& cross,
                                               bool& on, int& par)
{
    const bool have = k < nu;
    const int2 a = have ? u[k] : make_int2(0, 0);
    const int2 b = have ? u[k + 1 == nu ? 0 : k + 1] : make_int2(0, 0);
    for (int g = 0; g < nw; ++g) {
        const int2 c = w[g];
        const int2 d = w[g + 1 == nw ? 0 : g + 1];
        if (!have) continue;
        const int o1 = orient_sign64(a.x, a.y, b.x, b.y, c.x, c.y), o2 = orient_sign64(a.x, a.y, b.x, b.y, d.x, d.y);
        const int o3 = orient_sign64(c.x, c.y, d.x, d.y, a.x, a.y), o4 = orient_sign64(c.x, c.y, d.x, d.y, b.x, b.y);
        cross |= (o1 * o2 < 0) & (o3 * o4 < 0);
        on |= (o3 == 0) & (a.x >= min(c.x, d.x)) & (a.x <= max(c.x, d.x)) & (a.y >= min(c.y, d.y)) &
              (a.y <= max(c.y, d.y));
        const int lo_y = min(c.y, d.y), hi_y = max(c.y, d.y);
        if (lo_y <= a.y && a.y < hi_y) {
            const int2 l = c.y < d.y ? c : d, h = c.y < d.y ? d : c;
            par ^= ((long long)(a.x - l.x) * (h.y - l.y) < (long long)(a.y - l.y) * (h.x - l.x)) ? 1 : 0;
        }
    }
}

// ST_Touches by the stated rule: no proper edge crossing, no vertex of one strictly within the
// other (even-odd, off its boundary), some vertex of one on an edge of the other. One warp per pair;
// 1 / 0, 0xff for invalid indices. O(n_p n_q) per pair.
__global__ void __launch_bounds__(256) k_touches(const int32_t* pa, const int32_t* pb, long long n, long long nA,
                                                 long long nB, const int64_t* offA, const int32_t* xyA,
                                                 const int64_t* offB, const int32_t* xyB, uint8_t* out)
{
    const int lane = threadIdx.x & 31;
    const long long nwarps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += nwarps) {
        const int ia = pa[i], ib = pb[i];
        if (ia < 0 || ia >= nA || ib < 0 || ib >= nB) {
            if (lane == 0) out[i] = 0xff;
            continue;
        }
        const int2* p = reinterpret_cast<const int2*>(xyA) + offA[ia];
        const int2* q = reinterpret_cast<const int2*>(xyB) + offB[ib];
        const int np = (int)(offA[ia + 1] - offA[ia]), nq = (int)(offB[ib + 1] - offB[ib]);
        bool cross = false, inside = false, on_any = false;
        for (int side = 0; side < 2 && !cross && !inside; ++side) {       // warp-uniform conditions
            const int2* u = side ? q : p;
            const int2* w = side ? p : q;
            const int nu = side ? nq : np, nw = side ? np : nq;
            for (int base = 0; base < nu; base += 32) {
                bool cr = false, on = false;
                int par = 0;
                vertex_vs_ring(u, nu, base + lane, w, nw, cr, on, par);
                const bool have = base + lane < nu;
                cross |= __any_sync(kFull, have && cr);
                inside |= __any_sync(kFull, have && !on && par);
                on_any |= __any_sync(kFull, have && on);
                if (cross || inside) break;
            }
        }
        if (lane == 0) out[i] = (uint8_t)((!cross && !inside && on_any) ? 1 : 0);
    }
}

// ----------------------------------------------------------------------------------------------
// Integer ALU issue rate (the denominator of the pair-area kernels' roofline): every thread runs
// kAluChains independent chains of int32 multiply-add, three-input XOR and three-input add, each
// statement one instruction of the integer units (IMAD, LOP3, IADD3 classes); kAluPerIter of them per
// iteration. The operands depend on the thread and on `seed`, and the result is stored only when it
// equals `seed`, so nothing can be folded away or skipped.
// ----------------------------------------------------------------------------------------------
constexpr int kAluChains = 12;
constexpr int kAluPerIter = 24;     // statements per loop iteration (two rounds over the chains)

__global__ void __launch_bounds__(256) k_alu_probe(int iters, uint32_t seed, uint32_t* sink)
{
    uint32_t r[kAluChains];
#pragma unroll
    for (int k = 0; k < kAluChains; ++k) r[k] = (threadIdx.x + 977u * blockIdx.x) * (2u * k + 1u) ^ (seed + k);
    const uint32_t m = seed | 1u;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int round = 0; round < 2; ++round) {
#pragma unroll
            for (int k = 0; k < kAluChains; k += 3) {
                r[k] = r[k] * m + r[k + 1];                     // multiply-add
                r[k + 1] = r[k + 1] ^ r[k + 2] ^ r[k];          // three-input XOR
                r[k + 2] = r[k + 2] + r[k] + r[k + 1];          // three-input add
            }
        }
    }
    uint32_t x = 0;
#pragma unroll
    for (int k = 0; k < kAluChains; ++k) x ^= r[k];
    if (x == seed) sink[0] = x;
}

// ----------------------------------------------------------------------------------------------
// a6: Jaccard reductions (exact integer sums; ratios summed in 128-bit fixed point, scale 2^84)
// ----------------------------------------------------------------------------------------------
struct JPart {
    unsigned long long si, su, nz, fx_lo, fx_hi;
};

// Fixed-point scale of the J' sum. A ratio r = inter/union with 0 < inter <= union < 2^31 lies in
// [2^-31, 1], so its last significand bit weighs at least 2^-83 and r * 2^84 is an integer below
// 2^85: the sum of fewer than 2^43 ratios is exact in 128 bits (kJaccardMaxPairs).
constexpr int kJScale = 84;
constexpr long long kJaccardMaxPairs = 1LL << 43;

// floor(N / d) and N - d floor(N / d) for d in [2^31, 2^32) and N < 2^64 with N / d < 2^33, in
// exact integer arithmetic: an fp32 estimate of the quotient (relative error below 2^-22), the exact
// remainder of that estimate (differences wrap modulo 2^64 but stay below 2^43 in magnitude, so
// their signed reading is right), one fp32 correction from the remainder (error below 2), and the
// last steps by comparison.
__device__ __forceinline__ unsigned long long divmod_norm(unsigned long long N, unsigned d, unsigned long long& rem)
{
    const float rd = __frcp_rn((float)d);
    unsigned long long q = (unsigned long long)(__ull2float_rn(N) * rd);
    long long r = (long long)(N - q * (unsigned long long)d);
    const long long c = (long long)(__ll2float_rn(r) * rd);
    q += (unsigned long long)c;
    r -= c * (long long)d;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (r < 0) { --q; r += d; }
        if (r >= (long long)d) { ++q; r -= d; }
    }
    rem = (unsigned long long)r;
    return q;
}

// r = inter/union as an IEEE double (rounded to nearest, ties to even), returned as r * 2^kJScale
// (exact, see above). For 0 < inter <= union < 2^31 the quotient is formed in integers: with both
// shifted to 32 bits (in, un in [2^31, 2^32)), r = (in / un) 2^(a - b) for their top-bit positions a,
// b; its exponent e is a - b, or a - b - 1 when in < un; its 53-bit significand is
// M = floor(in 2^t / un) with t = 52 + (a - b - e), by two divisions of a 64-bit by a 32-bit number
// (the first quotient's remainder shifted up 32 bits for the second), and the remainder R rounds it
// (up when 2R > un, or 2R = un and M is odd). Then r 2^kJScale = M 2^(e + 32). Other inputs take the
// double division.
__device__ __forceinline__ unsigned __int128 ratio_fixed(long long inter, long long uni)
{
    if (inter > 0 && inter <= uni && uni < (1LL << 31)) {
        const unsigned i = (unsigned)inter, u = (unsigned)uni;
        const int a = 31 - __clz(i), b = 31 - __clz(u);
        const unsigned in = i << (31 - a), un = u << (31 - b);
        const int e = a - b - (in < un ? 1 : 0);
        const int t = 52 + (a - b - e);                          // 52 or 53
        unsigned long long r1, r2;
        const unsigned long long q1 = divmod_norm((unsigned long long)in << (t - 32), un, r1);
        const unsigned long long q2 = divmod_norm(r1 << 32, un, r2);
        unsigned long long M = (q1 << 32) + q2;                  // in [2^52, 2^53)
        if (2 * r2 > un || (2 * r2 == un && (M & 1))) ++M;       // may reach 2^53: still exact
        return (unsigned __int128)M << (e + 32);
    }
    const double r = __ddiv_rn((double)inter, (double)uni);
    const unsigned long long bits = (unsigned long long)__double_as_longlong(r);
    const int ex = (int)((bits >> 52) & 0x7ff);
    const unsigned long long man = (bits & ((1ull << 52) - 1)) | (1ull << 52);
    const int sh = min(max(ex - 1075 + kJScale, 0), 74);   // 1 .. 32 whenever 0 < inter <= union < 2^31
    return (unsigned __int128)man << sh;
}

__device__ __forceinline__ unsigned long long shfl_down_u64(unsigned long long v, int o)
{
    return __shfl_down_sync(kFull, v, o);
}

__global__ void __launch_bounds__(256) k_jaccard_partial(const int64_t* __restrict__ inter,
                                                         const int64_t* __restrict__ uni, long long n,
                                                         JPart* parts)
{
    unsigned long long si = 0, su = 0, nz = 0;
    unsigned __int128 fx = 0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long in = inter[i];
        if (in > 0) {
            const long long un = uni[i];
            si += (unsigned long long)in;
            su += (unsigned long long)un;
            nz += 1;
            fx += ratio_fixed(in, un);
        }
    }
    unsigned long long lo = (unsigned long long)fx, hi = (unsigned long long)(fx >> 64);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        si += shfl_down_u64(si, o);
        su += shfl_down_u64(su, o);
        nz += shfl_down_u64(nz, o);
        const unsigned long long l2 = shfl_down_u64(lo, o), h2 = shfl_down_u64(hi, o);
        const unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    __shared__ JPart sh[8];
    const int warp = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) sh[warp] = JPart{si, su, nz, lo, hi};
    __syncthreads();
    if (threadIdx.x == 0) {
        JPart t = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            t.si += sh[w].si; t.su += sh[w].su; t.nz += sh[w].nz;
            const unsigned long long nl = t.fx_lo + sh[w].fx_lo;
            t.fx_hi += sh[w].fx_hi + (nl < t.fx_lo ? 1ull : 0ull);
            t.fx_lo = nl;
        }
        parts[blockIdx.x] = t;
    }
}

struct JaccardOut {          // mirrors sccg_jaccard_result
    long long sum_inter, sum_union, n_nonzero, n_pairs;
    double J, Jprime;
};

// Round a nonnegative 128-bit integer to the nearest double (ties to even) and scale by 2^e.
__device__ __forceinline__ double u128_to_double_scaled(unsigned __int128 s, int e)
{
    if (s == 0) return 0.0;
    const unsigned long long hi = (unsigned long long)(s >> 64), lo = (unsigned long long)s;
    const int top = hi ? 127 - __clzll((long long)hi) : 63 - __clzll((long long)lo);
    unsigned long long m;
    int sh = 0;
    if (top <= 52) {
        m = lo;
    } else {
        sh = top - 52;
        m = (unsigned long long)(s >> sh);
        const unsigned __int128 rem = s & ((((unsigned __int128)1) << sh) - 1);
        const unsigned __int128 half = ((unsigned __int128)1) << (sh - 1);
        if (rem > half || (rem == half && (m & 1ull))) {
            m += 1;
            if (m == (1ull << 53)) { m >>= 1; sh += 1; }
        }
    }
    // m < 2^53 converts exactly; the power of two is built from its exponent bits
    const int pe = sh + e;
    const double p2 = __longlong_as_double((long long)(1023 + pe) << 52);
    return (double)m * p2;
}

// Combine the partial sums (one CTA of 256 threads) and form J and J'.
__global__ void __launch_bounds__(256) k_jaccard_final(const JPart* parts, int nparts, long long n_pairs,
                                                       JaccardOut* out)
{
    unsigned long long si = 0, su = 0, nz = 0, lo = 0, hi = 0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) {
        const JPart p = parts[i];
        si += p.si; su += p.su; nz += p.nz;
        const unsigned long long nl = lo + p.fx_lo;
        hi += p.fx_hi + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        si += shfl_down_u64(si, o);
        su += shfl_down_u64(su, o);
        nz += shfl_down_u64(nz, o);
        const unsigned long long l2 = shfl_down_u64(lo, o), h2 = shfl_down_u64(hi, o);
        const unsigned long long nl = lo + l2;
        hi = hi + h2 + (nl < lo ? 1ull : 0ull);
        lo = nl;
    }
    __shared__ JPart sh[8];
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = JPart{si, su, nz, lo, hi};
    __syncthreads();
    if (threadIdx.x != 0) return;
    JPart t = sh[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
        t.si += sh[w].si; t.su += sh[w].su; t.nz += sh[w].nz;
        const unsigned long long nl = t.fx_lo + sh[w].fx_lo;
        t.fx_hi += sh[w].fx_hi + (nl < t.fx_lo ? 1ull : 0ull);
        t.fx_lo = nl;
    }
    JaccardOut r;
    r.sum_inter = (long long)t.si;
    r.sum_union = (long long)t.su;
    r.n_nonzero = (long long)t.nz;
    r.n_pairs = n_pairs;
    if (t.nz == 0) {
        r.J = 0.0; r.Jprime = 0.0;
    } else {
        r.J = __ddiv_rn(__ll2double_rn((long long)t.si), __ll2double_rn((long long)t.su));
        const unsigned __int128 s = ((unsigned __int128)t.fx_hi << 64) | t.fx_lo;
        const double sum = u128_to_double_scaled(s, -kJScale);
        r.Jprime = __ddiv_rn(sum, __ll2double_rn((long long)t.nz));
    }
    *out = r;
}

// ----------------------------------------------------------------------------------------------
// Segmented helpers: batch assembly and per-segment Jaccard (jobs of a serving batch, tiles)
// ----------------------------------------------------------------------------------------------

// One CTA per segment s: copies src[seg_src[s] .. seg_src[s] + len) to dst[seg_dst[s] ..), where
// len = seg_dst[s+1] - seg_dst[s].
__global__ void __launch_bounds__(256) k_gather_pairs(const int32_t* __restrict__ src_a,
                                                      const int32_t* __restrict__ src_b,
                                                      const int64_t* __restrict__ seg_src,
                                                      const int64_t* __restrict__ seg_dst, int nseg,
                                                      int32_t* __restrict__ dst_a, int32_t* __restrict__ dst_b)
{
    for (int sgm = blockIdx.x; sgm < nseg; sgm += gridDim.x) {
        const long long s0 = seg_src[sgm], d0 = seg_dst[sgm], len = seg_dst[sgm + 1] - d0;
        for (long long i = threadIdx.x; i < len; i += blockDim.x) {
            dst_a[d0 + i] = src_a[s0 + i];
            dst_b[d0 + i] = src_b[s0 + i];
        }
    }
}

// One CTA (256 threads) per segment: the Jaccard reductions of pairs seg_off[s] .. seg_off[s+1]-1,
// with the same exact sums as k_jaccard_partial / k_jaccard_final.
__global__ void __launch_bounds__(256) k_jaccard_segments(const int64_t* __restrict__ inter,
                                                          const int64_t* __restrict__ uni,
                                                          const int64_t* __restrict__ seg_off, int nseg,
                                                          JaccardOut* out)
{
    __shared__ JPart sh[8];
    for (int sgm = blockIdx.x; sgm < nseg; sgm += gridDim.x) {
        const long long lo_i = seg_off[sgm], hi_i = seg_off[sgm + 1];
        unsigned long long si = 0, su = 0, nz = 0;
        unsigned __int128 fx = 0;
        for (long long i = lo_i + threadIdx.x; i < hi_i; i += blockDim.x) {
            const long long in = inter[i];
            if (in > 0) {
                const long long un = uni[i];
                si += (unsigned long long)in;
                su += (unsigned long long)un;
                nz += 1;
                fx += ratio_fixed(in, un);
            }
        }
        unsigned long long lo = (unsigned long long)fx, hi = (unsigned long long)(fx >> 64);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            si += shfl_down_u64(si, o);
            su += shfl_down_u64(su, o);
            nz += shfl_down_u64(nz, o);
            const unsigned long long l2 = shfl_down_u64(lo, o), h2 = shfl_down_u64(hi, o);
            const unsigned long long nl = lo + l2;
            hi = hi + h2 + (nl < lo ? 1ull : 0ull);
            lo = nl;
        }
        if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = JPart{si, su, nz, lo, hi};
        __syncthreads();
        if (threadIdx.x == 0) {
            JPart t = sh[0];
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
                t.si += sh[w].si; t.su += sh[w].su; t.nz += sh[w].nz;
                const unsigned long long nl = t.fx_lo + sh[w].fx_lo;
                t.fx_hi += sh[w].fx_hi + (nl < t.fx_lo ? 1ull : 0ull);
                t.fx_lo = nl;
            }
            JaccardOut r;
            r.sum_inter = (long long)t.si;
            r.sum_union = (long long)t.su;
            r.n_nonzero = (long long)t.nz;
            r.n_pairs = hi_i - lo_i;
            if (t.nz == 0) {
                r.J = 0.0; r.Jprime = 0.0;
            } else {
                r.J = __ddiv_rn(__ll2double_rn((long long)t.si), __ll2double_rn((long long)t.su));
                const unsigned __int128 s = ((unsigned __int128)t.fx_hi << 64) | t.fx_lo;
                r.Jprime = __ddiv_rn(u128_to_double_scaled(s, -kJScale), __ll2double_rn((long long)t.nz));
            }
            out[sgm] = r;
        }
        __syncthreads();
    }
}

}  // namespace sccg
