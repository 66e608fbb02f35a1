// Exact pixel area ||p|| of one polygon by rows (a2, the pixel-count counterpart of the shoelace
// area of Sec. 3.2): for every pixel row, the crossing positions of the edges that straddle it
// give the inside pixels directly, so the cost grows with the edges per row, not with the area.
//
// Row y, an edge straddling it (lower endpoint (xl, ylo), dy > 0, dx), and a base column xb at or
// left of every vertex: pixel xb + t (t >= 0) is crossed by the edge iff
//   2 t dy < N,  N = (2 (y - ylo) + 1) dx - (2 (xb - xl) + 1) dy      (same rule as the strips)
// so the edge crosses exactly the first c = #{t >= 0 : 2 t dy < N} pixels right of xb
// (c = 0 if N <= 0, else ceil(N / (2 dy))). With the row's k values sorted, s_0 <= ... <= s_{k-1}
// (k is even: a closed ring meets a row line an even number of times), pixel xb + t is crossed
// k - #{j : s_j <= t} times, which is odd exactly on [s_0, s_1), [s_2, s_3), ... The row's count
// is therefore  sum_m (s_{2m+1} - s_{2m})  =  sum_i (+1 if rank_i is odd else -1) * c_i  with
// ranks taken in any order consistent with the values (equal values cancel whatever their order).
// Pixels left of xb are crossed by all k edges (even) and are outside.
//
// All products stay within int32 under the set limits (|extent| <= 16384): |N| < 2^30.
#pragma once
#include <cstdint>

#include "pixelbox.cuh"

namespace sccg {

constexpr int kScanEntries = 1024;   // (edge, row) crossing values held per pass

struct alignas(16) ScanSmem {
    int cnt[32];                 // per-row crossing counts of the current 32-row band
    int off[33];                 // their exclusive prefix within the current row group
    int val[kScanEntries];       // crossing values c, grouped by row
};

// Inside pixels of one row from its k crossing values (one lane).
__device__ __forceinline__ uint32_t row_inside(const int* val, int k)
{
    int s = 0;
    for (int i = 0; i < k; ++i) {
        const int vi = val[i];
        int r = 0;
        for (int j = 0; j < k; ++j) {
            const int vj = val[j];
            r += (vj < vi) | ((vj == vi) & (j < i));
        }
        s += (r & 1) ? vi : -vi;
    }
    return (uint32_t)s;
}

// Inside pixels of row y over columns [x0, x1) from the whole ring, 32 pixels at a time with the
// edges spread over the lanes (used for a row crossed by more edges than a pass holds). Whole warp.
__device__ __forceinline__ uint32_t row_direct(const int2* v, int nv, int y, int x0, int x1, int lane)
{
    uint32_t total = 0;
    for (int xs = x0; xs < x1; xs += 32) {
        uint32_t par = 0;
        for (int base = 0; base < nv; base += 32) {
            const int e = base + lane;
            if (e < nv) {
                const int f = (e + 1 == nv) ? 0 : e + 1;
                int2 a = v[e];
                int2 b = v[f];
                if (b.y < a.y) { const int2 t = a; a = b; b = t; }
                const int dy = b.y - a.y;
                if (y >= a.y && y < b.y) {
                    const int c = min(crossing_count(a.y, dy, b.x - a.x, a.x, y, xs), 32);
                    par ^= __funnelshift_lc(0xffffffffu, 0u, (unsigned)c);
                }
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) par ^= __shfl_xor_sync(kFull, par, o);
        total += __popc(par & __funnelshift_lc(0xffffffffu, 0u, (unsigned)min(32, x1 - xs)));
    }
    return total;
}

// Edge sources for the row counting: the edges of a ring (closing edge included), or edge records
// {ylo, dy, dx, xl} (a band of a band index). get() returns edge k with its lower endpoint first.
struct RingEdges {
    const int2* v;
    int n;
    __device__ __forceinline__ void get(int k, int& ylo, int& dy, int& dx, int& xl) const
    {
        const int f = (k + 1 == n) ? 0 : k + 1;
        int2 a = v[k];
        int2 b = v[f];
        if (b.y < a.y) { const int2 t = a; a = b; b = t; }
        ylo = a.y; dy = b.y - a.y; dx = b.x - a.x; xl = a.x;
    }
};

struct RecordEdges {
    const int4* e;
    int n;
    __device__ __forceinline__ void get(int k, int& ylo, int& dy, int& dx, int& xl) const
    {
        const int4 r = e[k];
        ylo = r.x; dy = r.y; dx = r.z; xl = r.w;
    }
};

// This lane's share of the inside pixels of rows b0 .. b0 + nrows - 1 (nrows <= 32), over columns
// [x0, x1), from the edges of `src`, which must include every edge of the ring that straddles one of
// those rows (more edges are harmless). A row crossed by more edges than one pass holds is counted
// from the whole ring (row_direct). Whole warp, converged.
template <bool COUNT, class Edges>
__device__ __forceinline__ uint32_t band_rows(const Edges src, int b0, int nrows, int x0, int x1, const int2* ring,
                                              int nring, ScanSmem& S, int lane, WorkCounters& wc)
{
    uint32_t acc = 0;
    S.cnt[lane] = 0;
    __syncwarp();
    for (int base = 0; base < src.n; base += 32) {          // per-row counts, one edge per lane
        const int e = base + lane;
        if (e < src.n) {
            int ylo, dy, dx, xl;
            src.get(e, ylo, dy, dx, xl);
            const int r1 = min(ylo + dy, b0 + nrows) - b0;
            for (int q = max(ylo, b0) - b0; q < r1; ++q) atomicAdd(&S.cnt[q], 1);
        }
    }
    __syncwarp();
    const int c = S.cnt[lane];
    int r = 0;
    while (r < nrows) {
        // the longest run of rows from r whose crossing values fit one pass
        const int cm = (lane >= r && lane < nrows) ? c : 0;
        int incl = cm;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        const unsigned fit = __ballot_sync(kFull, lane >= r && lane < nrows && incl <= kScanEntries);
        const int r2 = fit ? 32 - __clz(fit) : r;
        if (r2 == r) {
            // a single row with more crossings than a pass holds
            const uint32_t t = row_direct(ring, nring, b0 + r, x0, x1, lane);
            if (lane == 0) acc += t;
            r += 1;
            continue;
        }
        S.off[lane] = incl - cm;
        S.cnt[lane] = 0;          // fill cursor
        __syncwarp();
        for (int base = 0; base < src.n; base += 32) {      // crossing values, one edge per lane
            const int e = base + lane;
            if (e < src.n) {
                int ylo, dy, dx, xl;
                src.get(e, ylo, dy, dx, xl);
                const int q1 = min(ylo + dy, b0 + r2) - b0;
                for (int q = max(ylo, b0 + r) - b0; q < q1; ++q)
                    S.val[S.off[q] + atomicAdd(&S.cnt[q], 1)] = crossing_count(ylo, dy, dx, xl, b0 + q, x0);
            }
        }
        __syncwarp();
        if (lane >= r && lane < r2) {
            acc += row_inside(S.val + S.off[lane], c);
            if (COUNT) {
                wc.scan_entries += (unsigned long long)c;
                wc.scan_pairs += (unsigned long long)c * c;
            }
        }
        __syncwarp();
        r = r2;
    }
    return acc;
}

// ||p|| over the pixel window [x0, x1) x [y0, y1) (x0 at or left of every vertex), band by band
// of 32 rows, one lane per row. Returns the warp-wide count (same in every lane). Whole warp,
// converged; every loop before a collective has a warp-uniform trip count.
template <bool COUNT>
__device__ __forceinline__ uint32_t area_scan(const int2* v, int nv, int x0, int y0, int x1, int y1, ScanSmem& S,
                                              int lane, WorkCounters& wc)
{
    uint32_t acc = 0;
    for (int b0 = y0; b0 < y1; b0 += 32)
        acc += band_rows<COUNT>(RingEdges{v, nv}, b0, min(32, y1 - b0), x0, x1, v, nv, S, lane, wc);
    return warp_sum(acc);
}

}  // namespace sccg
