// PixelBox device core for sm_103a: exact pixel counting by sampling-box subdivision (Sec. 3.2)
// with per-pixel ray casting on mixed boxes (Sec. 3.1), one warp per polygon pair.
//
// Pixel model. Pixel (x, y) is [x, x+1) x [y, y+1) with centre (x + 1/2, y + 1/2). It is inside
// polygon p when the ray from its centre towards +x crosses p's boundary an odd number of times
// (Fig. 4b). In doubled coordinates the centre (2x+1, 2y+1) is odd and every vertex even, so the ray
// never meets a vertex; an edge with lower endpoint (xl, ylo) and upper (xl+dx, ylo+dy), dy > 0,
// straddles row y iff ylo <= y < ylo+dy and is crossed iff its x at the row is strictly right of
// the centre:  (2(x - xl) + 1) * dy  <  (2(y - ylo) + 1) * dx.   (centre on the edge: not counted)
//
// Everything below is integer-exact in int32 for coordinates within +-2^28 and polygon bounding
// boxes at most 16384 px wide and high (checked when the set is prepared): every product has one
// factor bounded by the polygon's extent and the other by twice it.
//
// Style: every helper takes plain pointers and values (no structs of pointers passed by reference,
// no lambdas), warp collectives are shuffles executed by the converged warp, and loops that
// precede a collective have warp-uniform trip counts.
#pragma once
#include <cstdint>

namespace sccg {

constexpr unsigned kFull = 0xffffffffu;

struct WorkCounters {          // algorithmic work, accumulated only by the counting instantiation
    unsigned long long strip_edges;   // (32-pixel row strip, edge) evaluations
    unsigned long long pixel_edges;   // (valid pixel, edge) point-in-polygon tests inside those
    unsigned long long box_edges;     // (sampling box, edge) classifications
    unsigned long long boxes;         // sampling boxes classified (per polygon)
    unsigned long long row_entries;   // (edge, row) crossings XORed into leaf parity words
    unsigned long long row_edges;     // (row, 32-pixel word) parity words of leaf windows reduced
    unsigned long long scan_entries;  // (edge, row) crossing values of the by-rows area
    unsigned long long scan_pairs;    // crossing-value comparisons ranking them
    unsigned long long leaf_pixels;   // (pixel, polygon) memberships decided one pixel at a time
    unsigned long long window_pixels; // pixels of the windows counted (pairs' windows or items)
    unsigned long long raster_out;    // pixel raster words written (sets that keep rasters)
    unsigned long long raster_and;    // (row, word) ANDs of two rasters over pairs' windows
};

// Warp-wide reductions (redux.sync: one instruction each). Whole warp, converged.
__device__ __forceinline__ int warp_min(int v) { return __reduce_min_sync(kFull, v); }
__device__ __forceinline__ int warp_max(int v) { return __reduce_max_sync(kFull, v); }
__device__ __forceinline__ unsigned warp_sum(unsigned v) { return __reduce_add_sync(kFull, v); }

// Stage edges [e0, e0 + cnt) of the ring v[0..nv) into E/R (whole warp; uniform trip count).
// Edge record: int4 {ylo, dy, dx, xl} (lower endpoint first; a horizontal edge keeps its first
// endpoint and dy = 0) plus R = RN(1 / (2 dy)).
__device__ __forceinline__ void stage_edges(const int2* v, int nv, int e0, int cnt, int4* E, float* R,
                                            int lane)
{
    for (int base = 0; base < cnt; base += 32) {
        const int i = base + lane;
        if (i < cnt) {
            const int e = e0 + i;
            const int f = (e + 1 == nv) ? 0 : e + 1;
            int2 a = v[e];
            int2 b = v[f];
            if (b.y < a.y) { const int2 t = a; a = b; b = t; }
            const int dy = b.y - a.y;
            E[i] = make_int4(a.y, dy, b.x - a.x, a.x);
            R[i] = dy > 0 ? __frcp_rn((float)(2 * dy)) : 0.0f;
        }
    }
}

// Stage, from the ring v[0..nv), only the edges that can affect a pixel of the window
// [x0, x1) x [y0, y1): those with ylo < y1, yhi > y0 and max x > x0. Any other edge lies wholly on
// or below the line y = y0, on or above y = y1, or on or left of x = x0, while every pixel centre
// of the window, and every centre rectangle R of a box inside it, lies strictly inside those three
// lines: such an edge straddles no row of the window, is never right of a centre in it and meets
// no R. Dropping it changes no crossing parity and no box position, so every count over the
// window is unchanged. Returns the number of kept edges (warp-uniform); only the first `cap` are
// stored, so a return value above `cap` means the caller must use the whole ring instead.
//
// Windows of at most 64 rows also drop the edges lying wholly on or right of x = x1: every pixel
// centre of the window is strictly left of such an edge, so it crosses all of them in each row it
// straddles and meets no box. Its effect is recorded instead in `flip` (bit r: the edges dropped
// this way flip every pixel of row y0 + r an odd number of times), which the pixelization and the
// box positions add back (row_flip).
__device__ __forceinline__ unsigned long long row_span_mask(int r0, int r1)    // bits r0 .. r1-1, 0 <= r0 <= r1 <= 64
{
    const unsigned long long hi = r1 >= 64 ? ~0ull : ((1ull << r1) - 1ull);
    const unsigned long long lo = (1ull << r0) - 1ull;
    return hi & ~lo;
}

__device__ __forceinline__ int stage_culled(const int2* v, int nv, int x0, int y0, int x1, int y1, int4* E,
                                            float* R, int cap, int lane, bool right, unsigned long long& flip)
{
    const bool rows64 = right && y1 - y0 <= 64;
    int cnt = 0;
    unsigned long long fl = 0;
    for (int base = 0; base < nv; base += 32) {
        const int e = base + lane;
        bool keep = false;
        int4 rec = make_int4(0, 0, 0, 0);
        float rc = 0.0f;
        if (e < nv) {
            const int f = (e + 1 == nv) ? 0 : e + 1;
            int2 a = v[e];
            int2 b = v[f];
            if (b.y < a.y) { const int2 t = a; a = b; b = t; }
            const int dy = b.y - a.y;
            keep = (a.y < y1) & (b.y > y0) & (max(a.x, b.x) > x0);
            if (keep && rows64 && min(a.x, b.x) >= x1) {
                keep = false;
                fl ^= row_span_mask(max(a.y, y0) - y0, min(b.y, y1) - y0);
            }
            rec = make_int4(a.y, dy, b.x - a.x, a.x);
            rc = dy > 0 ? __frcp_rn((float)(2 * dy)) : 0.0f;
        }
        const unsigned m = __ballot_sync(kFull, keep);
        const int pos = cnt + __popc(m & ((1u << lane) - 1u));
        if (keep && pos < cap) {
            E[pos] = rec;
            R[pos] = rc;
        }
        cnt += __popc(m);
    }
    if (right) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) fl ^= __shfl_xor_sync(kFull, fl, o);
    }
    flip = fl;
    return cnt;
}

// All ones when the dropped right-side edges flip row y of a window starting at row wy0.
__device__ __forceinline__ uint32_t row_flip(unsigned long long flip, int y, int wy0)
{
    const int r = y - wy0;
    return (r >= 0 && r < 64 && ((flip >> r) & 1ull)) ? 0xffffffffu : 0u;
}

// Parity bitmask of the 32 pixels (x0 + k, y), k = 0..31, against `cnt` staged edges.
//
// For a straddling edge, pixel x0 + k is crossed iff 2k*dy < D with
//   D = (2(y - ylo) + 1) dx - (2(x0 - xl) + 1) dy,
// so the crossed pixels of the strip are its first c = #{k in [0,32): 2k dy < D} pixels and the
// edge flips the parity of a prefix mask. c = 0 if D <= 0, else min(32, ceil(D / (2 dy))).
// The quotient is formed in fp32 from Dc = clamp(D, 0, 64 dy) (< 2^21, exact in fp32) and the
// correctly rounded reciprocal R: q = fma(Dc, R, -2^-17) carries a relative error below 2^-23
// (|abs error| < 2^-18 for quotients <= 32), while a non-integer quotient lies at least
// 1/(2 dy) >= 2^-15 from an integer; the -2^-17 offset keeps exact integers from rounding up.
// Hence ceil(q) is exact. ceil is taken by an upward-rounded add of 1.5 * 2^23 (unit spacing there).
__device__ __forceinline__ uint32_t strip_parity(const int4* E, const float* R, int cnt, int y, int x0)
{
    const int sx = 2 * x0 + 1;
    uint32_t par = 0;
#pragma unroll 4
    for (int i = 0; i < cnt; ++i) {
        const int4 ed = E[i];
        const float rc = R[i];
        const int t = y - ed.x;
        const bool st = (unsigned)t < (unsigned)ed.y;
        const int D = (2 * t + 1) * ed.z - (sx - 2 * ed.w) * ed.y;
        const int Dc = min(max(D, 0), ed.y << 6);
        const float f = __int_as_float(Dc | 0x4B000000) - 8388608.0f;
        const float q = __fmaf_rn(f, rc, -7.62939453125e-06f);
        const int c = __float_as_int(__fadd_ru(q, 12582912.0f)) - 0x4B400000;
        const uint32_t m = __funnelshift_lc(0xffffffffu, 0u, (unsigned)c);
        par ^= st ? m : 0u;
    }
    return par;
}

// Sampling-box position (Sec. 3.2, Lemma 1) of the pixel box [bx0, bx1) x [by0, by1) against `cnt`
// staged edges, accumulated into (meet, par).
//
// Exact reading of Lemma 1 for pixel centres: let R be the closed rectangle spanned by the box's
// pixel centres. If no edge meets R, all centres lie in one face of the polygon and none lies on
// an edge, so the box is inside or outside according to one centre (condition iii; here the centre
// of pixel (bx0, by0)). An edge meets R unless the rectangle and the segment are separated along
// x, along y, or along the segment's normal (all four corners strictly on one side of its line).
// A box met by any edge "hovers" and is refined or pixelized; this is conservative and exact.
__device__ __forceinline__ void box_scan(const int4* E, int cnt, int bx0, int by0, int bx1, int by1,
                                         bool& meet, uint32_t& par)
{
    const int cx = bx0 + bx1, cy = by0 + by1;          // centre of R, doubled coordinates
    const int hw = bx1 - bx0 - 1, hh = by1 - by0 - 1;  // half-extents of R, doubled coordinates
    const int sx = 2 * bx0 + 1;
    bool m = false;
    uint32_t p = 0;
#pragma unroll 2
    for (int i = 0; i < cnt; ++i) {
        const int4 ed = E[i];
        const int ylo = ed.x, dy = ed.y, dx = ed.z, xl = ed.w;
        const int xr = xl + dx;
        const int xmin = min(xl, xr), xmax = max(xl, xr);
        const bool bb = (xmax > bx0) & (xmin < bx1) & (ylo + dy > by0) & (ylo < by1);
        const int g = dx * (cy - 2 * ylo) - dy * (cx - 2 * xl);
        const int proj = dy * hw + abs(dx) * hh;
        m |= bb & (abs(g) <= proj);
        const int t = by0 - ylo;
        const bool st = (unsigned)t < (unsigned)dy;
        const bool cr = (sx - 2 * xl) * dy < (2 * t + 1) * dx;
        p ^= (uint32_t)(st & cr);
    }
    meet |= m;
    par ^= p;
}

// Strip parity against a whole polygon: its staged edges when resident (nv <= cap), else chunk by
// chunk re-staged into E/R. Whole warp, converged; `resident` is warp-uniform.
// `flip`: the resident polygon's row flip (row_flip) for row y.
template <bool COUNT>
__device__ __forceinline__ uint32_t poly_strip(const int2* v, int nv, bool resident, int4* E, float* R, int cap,
                                               int y, int x0, uint32_t flip, int lane, unsigned long long& cnt_edges)
{
    if (resident) {
        if (COUNT) cnt_edges += (unsigned long long)nv;
        return strip_parity(E, R, nv, y, x0) ^ flip;
    }
    uint32_t par = 0;
    for (int e0 = 0; e0 < nv; e0 += cap) {
        const int cnt = min(cap, nv - e0);
        __syncwarp();
        stage_edges(v, nv, e0, cnt, E, R, lane);
        __syncwarp();
        par ^= strip_parity(E, R, cnt, y, x0);
        if (COUNT) cnt_edges += (unsigned long long)cnt;
    }
    __syncwarp();
    return par;
}

// Box position against a whole polygon (resident or chunked, as above): 0 outside, 1 inside, 2 hover.
// `flip`: the resident polygon's row flip for row by0 (the reference centre's row).
template <bool COUNT>
__device__ __forceinline__ int poly_box(const int2* v, int nv, bool resident, int4* E, float* R, int cap,
                                        int bx0, int by0, int bx1, int by1, uint32_t flip, int lane,
                                        unsigned long long& cnt_edges)
{
    bool meet = false;
    uint32_t par = 0;
    if (resident) {
        par = flip & 1u;
        box_scan(E, nv, bx0, by0, bx1, by1, meet, par);
        if (COUNT) cnt_edges += (unsigned long long)nv;
    } else {
        for (int e0 = 0; e0 < nv; e0 += cap) {
            const int cnt = min(cap, nv - e0);
            __syncwarp();
            stage_edges(v, nv, e0, cnt, E, R, lane);
            __syncwarp();
            box_scan(E, cnt, bx0, by0, bx1, by1, meet, par);
            if (COUNT) cnt_edges += (unsigned long long)cnt;
        }
        __syncwarp();
    }
    return meet ? 2 : (int)(par & 1u);
}

// c = ceil(N / (2 dy)) for N > 0, else 0: the number of pixels xb, xb + 1, ... of row y crossed by
// an edge that straddles the row, with N = (2 (y - ylo) + 1) dx - (2 (xb - xl) + 1) dy (pixel xb + t is
// crossed iff 2 t dy < N, the rule of strip_parity). N / (2 dy) is the crossing's distance right of
// xb in pixels, at most 2^15 whenever xb is at or right of the polygon's minimum x minus its
// extent. The quotient is estimated in fp32 (relative error below 2^-22, absolute below 2^-7 at
// 2^15, so the estimate's ceiling is off by at most one) and corrected with exact integer products
// (< 2^31).
// r2 = RN(1 / (2 dy)) (the staged reciprocal).
__device__ __forceinline__ int crossing_count_r(int ylo, int dy, int dx, int xl, int y, int xb, float r2)
{
    const int N = (2 * (y - ylo) + 1) * dx - (2 * (xb - xl) + 1) * dy;
    const int d2 = 2 * dy;
    int c = (int)ceilf(__fmul_rn((float)N, r2));
    c += (c * d2 < N) ? 1 : 0;
    c -= ((c - 1) * d2 >= N) ? 1 : 0;
    return N <= 0 ? 0 : c;
}

__device__ __forceinline__ int crossing_count(int ylo, int dy, int dx, int xl, int y, int xb)
{
    return crossing_count_r(ylo, dy, dx, xl, y, xb, __frcp_rn((float)(2 * dy)));
}

// Parity words of a leaf window, one pass of up to 64 rows (pixelization in edge-major order).
// An edge that straddles row y crosses exactly the first c pixels of the row right of the window's
// left column x0 (c = crossing_count clamped to the window width W), so it flips those pixels'
// parity: words 0 .. c/32 - 1 entirely and the first c mod 32 pixels of word c/32. The whole-word
// flips are recorded as bit c/32 of F[r], the partial one XORed into P[r * nw + c/32]; the parity
// of pixel x0 + 32 j + k of row r is then bit k of
//   P[r * nw + j] ^ (all ones if F[r] has an odd number of bits above bit j).
// Windows are handled in pieces of at most kXorMaxWords words (992 px) so that c/32 fits F's bits.
constexpr int kXorWords = 256;
constexpr int kXorMaxWords = 31;
struct XorRows {
    unsigned F[64];
    unsigned P[kXorWords];
};

// Per-warp shared memory: edge buffers of the two polygons, their leaf parity words and the
// subdivision loop's state.
template <int CAP, int STK>
struct WarpSmem {
    int4 ep[CAP];
    int4 eq[CAP];
    float rp[CAP];
    float rq[CAP];
    XorRows xp;
    XorRows xq;
    uint2 stack[STK];     // pending sampling boxes (window-relative, packed with flags)
    uint2 leaf[32];       // boxes to pixelize in the current round, one slot per lane
    int loff[32];         // exclusive prefix of row strips over the leaf slots
};

// Flattened (edge, row) work: lane L holds an edge with cnt_L rows to visit and excl = the exclusive
// prefix sum of cnt over the lanes; entry t (0 <= t < total) belongs to the last lane whose excl is
// <= t (a lane with no rows never is: the next lane has the same offset). Binary search over the
// lanes by shuffles. Whole warp, converged.
__device__ __forceinline__ int flat_owner(int excl, int t)
{
    int own = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const int e = __shfl_sync(kFull, excl, own + s);   // own + s <= 31 throughout
        if (e <= t) own += s;
    }
    return own;
}

// Exclusive and total of cnt over the warp.
__device__ __forceinline__ int warp_excl(int cnt, int lane, int& total)
{
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    total = __shfl_sync(kFull, incl, 31);
    return incl - cnt;
}

// XOR the crossings of the `ne` staged edges with rows y0 .. y0 + nr - 1 into X (cleared), for
// columns x0 .. x0 + W - 1 (W <= 32 nw, nw <= kXorMaxWords). The (edge, row) crossings of each
// group of 32 edges are spread evenly over the lanes (warp prefix sum of the edges' row counts; each
// lane finds its crossing's edge by a binary search over the lanes' offsets), so a steep edge does
// not hold the warp. Whole warp, converged.
template <bool COUNT>
__device__ __forceinline__ void xor_rows(const int4* E, const float* R, int ne, int x0, int y0, int nr, int W, int nw,
                                         XorRows& X, int lane, unsigned long long& entries)
{
    for (int base = 0; base < ne; base += 32) {
        const int i = base + lane;
        int cnt = 0;
        if (i < ne) {
            const int4 ed = E[i];
            cnt = max(0, min(ed.x + ed.y, y0 + nr) - max(ed.x, y0));
        }
        int total;
        const int excl = warp_excl(cnt, lane, total);
        for (int t0 = 0; t0 < total; t0 += 32) {
            const int t = t0 + lane;
            const int own = flat_owner(excl, t);
            const int eo = __shfl_sync(kFull, excl, own);
            if (t < total) {
                const int4 ed = E[base + own];
                const int y = max(ed.x, y0) + (t - eo);
                const int c = min(crossing_count_r(ed.x, ed.y, ed.z, ed.w, y, x0, R[base + own]), W);
                const int q = c >> 5, rem = c & 31;
                const int r = y - y0;
                if (q) atomicXor(&X.F[r], 1u << q);
                if (rem) atomicXor(&X.P[r * nw + q], (1u << rem) - 1u);
            }
        }
        if (COUNT) entries += (unsigned long long)cnt;
    }
}

// The same XOR for edges held in registers instead of a staged buffer: each lane holds at most one
// edge {ylo, dy, dx, xl} (`has`), and an (edge, row) crossing's edge is fetched from its lane by
// shuffles. Edges with no pixel centre of the rows right of them (max x <= x0) are skipped, as the
// staging skips them. No buffer bounds the number of edges. Whole warp, converged; the trip count
// is warp-uniform.
__device__ __forceinline__ void xor_group(bool has, int ylo, int dy, int dx, int xl, int x0, int y0, int nr, int W,
                                          int nw, XorRows& X, int lane, unsigned long long& entries)
{
    int cnt = 0;
    if (has && max(xl, xl + dx) > x0) cnt = max(0, min(ylo + dy, y0 + nr) - max(ylo, y0));
    int total;
    const int excl = warp_excl(cnt, lane, total);
    if (total == 0) return;
    const float r2 = cnt > 0 ? __frcp_rn((float)(2 * dy)) : 0.0f;     // dy > 0 whenever cnt > 0
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        const int own = flat_owner(excl, t);
        const int eo = __shfl_sync(kFull, excl, own);
        const int oy = __shfl_sync(kFull, ylo, own), ody = __shfl_sync(kFull, dy, own);
        const int odx = __shfl_sync(kFull, dx, own), oxl = __shfl_sync(kFull, xl, own);
        const float orr = __shfl_sync(kFull, r2, own);
        if (t < total) {
            const int y = max(oy, y0) + (t - eo);
            const int c = min(crossing_count_r(oy, ody, odx, oxl, y, x0, orr), W);
            const int q = c >> 5, rem = c & 31;
            const int r = y - y0;
            if (q) atomicXor(&X.F[r], 1u << q);
            if (rem) atomicXor(&X.P[r * nw + q], (1u << rem) - 1u);
        }
    }
    entries += (unsigned long long)cnt;
}

// Parity word j of row r (see XorRows).
__device__ __forceinline__ uint32_t xor_word(const XorRows& X, int r, int nw, int j)
{
    return X.P[r * nw + j] ^ ((__popc(X.F[r] >> (j + 1)) & 1) ? 0xffffffffu : 0u);
}

// XOR the crossings of ring v[0..nv) with rows y0 .. y0 + nr - 1 (columns x0 .. x0 + W - 1) into X.
__device__ __forceinline__ void xor_stream_ring(const int2* v, int nv, int x0, int y0, int nr, int W, int nw,
                                                XorRows& X, int lane, unsigned long long& entries)
{
    for (int base = 0; base < nv; base += 32) {
        const int e = base + lane;
        int ylo = 0, dy = 0, dx = 0, xl = 0;
        if (e < nv) {
            const int f = (e + 1 == nv) ? 0 : e + 1;
            int2 p = v[e];
            int2 q = v[f];
            if (q.y < p.y) { const int2 t = p; p = q; q = t; }
            ylo = p.y; dy = q.y - p.y; dx = q.x - p.x; xl = p.x;
        }
        xor_group(e < nv, ylo, dy, dx, xl, x0, y0, nr, W, nw, X, lane, entries);
    }
}

// ||p|| over its window [x0, x1) x [y0, y1) (the polygon's MBR) as one leaf, edges streamed from the
// ring: pieces of up to 992 columns, passes of up to 64 rows, one lane per row in the reduction.
// Returns the warp-wide count. Whole warp, converged.
template <bool COUNT>
__device__ __forceinline__ uint32_t area_stream(const int2* v, int nv, int x0, int y0, int x1, int y1, XorRows& X,
                                                int lane, WorkCounters& wc)
{
    const int W = x1 - x0, H = y1 - y0;
    uint32_t acc = 0;
    if (COUNT && lane == 0) wc.window_pixels += (unsigned long long)W * H;
    for (int cx = 0; cx < W; cx += 32 * kXorMaxWords) {
        const int Wp = min(32 * kXorMaxWords, W - cx), nw = (Wp + 31) >> 5;
        const int nr = min(64, kXorWords / nw);
        for (int r0 = 0; r0 < H; r0 += nr) {
            const int nrr = min(nr, H - r0);
            __syncwarp();
            for (int k = lane; k < nrr; k += 32) X.F[k] = 0;
            for (int k = lane; k < nrr * nw; k += 32) X.P[k] = 0;
            __syncwarp();
            unsigned long long ce = 0;
            xor_stream_ring(v, nv, x0 + cx, y0 + r0, nrr, Wp, nw, X, lane, ce);
            __syncwarp();
            for (int k = lane; k < nrr; k += 32) {
                for (int j = 0; j < nw; ++j) {
                    const uint32_t in = __funnelshift_lc(0xffffffffu, 0u, (unsigned)min(32, Wp - 32 * j));
                    acc += __popc(in & xor_word(X, k, nw, j));
                }
                if (COUNT) {
                    wc.row_edges += (unsigned long long)nw;
                    wc.leaf_pixels += (unsigned long long)Wp;
                }
            }
            if (COUNT) wc.row_entries += ce;
        }
    }
    return warp_sum(acc);
}

// Box packing: window-relative coordinates (< 2^15) in 15 bits each; bit 15 of the low halves
// carries the "still needs testing against P / Q" flags.
__device__ __forceinline__ uint2 pack_box(int x0, int y0, int x1, int y1, int fl)
{
    return make_uint2((uint32_t)x0 | ((uint32_t)x1 << 16) | ((uint32_t)(fl & 1) << 15),
                      (uint32_t)y0 | ((uint32_t)y1 << 16) | ((uint32_t)(fl & 2) << 14));
}
__device__ __forceinline__ void unpack_box(uint2 b, int& x0, int& y0, int& x1, int& y1, int& fl)
{
    x0 = b.x & 0x7fff; x1 = (b.x >> 16) & 0x7fff;
    y0 = b.y & 0x7fff; y1 = (b.y >> 16) & 0x7fff;
    fl = ((b.x >> 15) & 1) | ((b.y >> 14) & 2);
}

// Choose a gx x gy split (gx * gy <= 32) of a w x h box that keeps the sub-boxes near square.
__device__ __forceinline__ void choose_split(int w, int h, int& gx, int& gy)
{
    int best = 0x7fffffff;
    gx = 1; gy = 32;
#pragma unroll
    for (int lg = 0; lg <= 5; ++lg) {
        const int ax = 1 << lg, ay = 32 >> lg;
        const long long u = (long long)w * ay, v = (long long)h * ax;
        const long long hi = u > v ? u : v, lo = u > v ? v : u;
        const int score = (int)min(hi / (lo > 0 ? lo : 1), (long long)0x7ffffffe);
        if (score < best) { best = score; gx = ax; gy = ay; }
    }
    gx = min(gx, w);
    gy = min(gy, h);
}

// The two polygons of a pair as seen by one warp (plain values).
struct PolyPair {
    const int2* vp; int np; bool rp_res;
    const int2* vq; int nq; bool rq_res;
    unsigned long long fp, fq;   // row flips of the edges dropped right of the window (buffers > 64 edges)
};

// Right-side culling (stage_culled) is used by the kernels whose buffers hold more than 64 edges,
// where large polygons' items carry many such edges; the 64-edge kernels keep them staged.
template <int CAP>
__device__ __forceinline__ uint32_t flip_of(unsigned long long f, int y, int wy0)
{
    if constexpr (CAP > 64) return row_flip(f, y, wy0);
    else return 0u;
}

// Pixelize the leaf boxes held in the lanes' slots (Algorithm 1's pixelization branch, done as
// 32-pixel row strips spread over the warp). Returns this lane's count of pixels inside every
// polygon its box still needs (UNION: inside any of them). Whole warp, converged.
template <bool TWO, bool COUNT, int CAP, int STK, bool UNION = false>
__device__ __forceinline__ uint32_t pixelize_leaves(const PolyPair pp, WarpSmem<CAP, STK>& S, int wx0, int wy0,
                                                    int lane, uint2 myleaf, bool have, WorkCounters& wc)
{
    int lx0, ly0, lx1, ly1, lfl;
    unpack_box(myleaf, lx0, ly0, lx1, ly1, lfl);
    const int nstr = have ? (ly1 - ly0) * ((lx1 - lx0 + 31) >> 5) : 0;
    int incl = nstr;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    const int total = __shfl_sync(kFull, incl, 31);
    S.leaf[lane] = myleaf;
    S.loff[lane] = incl - nstr;
    __syncwarp();
    uint32_t acc = 0;
    for (int k0 = 0; k0 < total; k0 += 32) {
        const int k = k0 + lane;
        const bool act = k < total;
        int j = 0;
#pragma unroll
        for (int s = 16; s > 0; s >>= 1)
            if (S.loff[j + s] <= k) j += s;
        int x0, y0, x1, y1, fl;
        unpack_box(S.leaf[j], x0, y0, x1, y1, fl);
        const int w = x1 - x0;
        const int chunks = max((w + 31) >> 5, 1);
        const int r = k - S.loff[j];
        const int row = chunks == 1 ? r : r / chunks;
        const int c = chunks == 1 ? 0 : r - row * chunks;
        const int y = wy0 + y0 + row;
        const int xs = wx0 + x0 + 32 * c;
        const int valid = min(32, w - 32 * c);
        const uint32_t vmask = act ? __funnelshift_lc(0xffffffffu, 0u, (unsigned)max(valid, 0)) : 0u;
        const bool needP = act && (fl & 1);
        const bool needQ = TWO && act && (fl & 2);
        uint32_t in = UNION ? 0u : vmask;
        unsigned long long ce = 0;
        if (__any_sync(kFull, needP)) {
            const uint32_t par = poly_strip<COUNT>(pp.vp, pp.np, pp.rp_res, S.ep, S.rp, CAP, y, xs,
                                                   flip_of<CAP>(pp.fp, y, wy0), lane, ce);
            if (needP) in = UNION ? (in | par) : (in & par);
            if (COUNT && needP) wc.pixel_edges += (unsigned long long)pp.np * valid;
        }
        if (TWO) {
            if (__any_sync(kFull, needQ)) {
                const uint32_t par = poly_strip<COUNT>(pp.vq, pp.nq, pp.rq_res, S.eq, S.rq, CAP, y, xs,
                                                       flip_of<CAP>(pp.fq, y, wy0), lane, ce);
                if (needQ) in = UNION ? (in | par) : (in & par);
                if (COUNT && needQ) wc.pixel_edges += (unsigned long long)pp.nq * valid;
            }
        }
        if (UNION) in &= vmask;
        if (COUNT) {
            wc.strip_edges += ce;
            wc.leaf_pixels += (unsigned long long)(needP ? valid : 0) + (needQ ? valid : 0);
        }
        acc += __popc(in);
    }
    __syncwarp();
    return acc;
}

// Count the pixels of the window [wx0, wx1) x [wy0, wy1) that lie inside P (and inside Q when TWO):
// PixelBox (Sec. 3.2-3.3). Boxes of at least T pixels are split into up to 32 sub-boxes, one per
// lane; each lane classifies its sub-box against the polygons the box still needs (a box inside P
// no longer needs P). Sub-boxes inside every needed polygon add their pixel count, sub-boxes
// outside any add nothing, mixed ones are pushed (>= T pixels) or pixelized (< T pixels).
// UNION (with TWO): count the pixels inside P or Q instead (the direct union of the PixelBox-NoSep
// variant, Sec. 5.2): a sub-box inside either polygon adds its pixels, one outside both adds
// nothing, and a polygon found outside a box is no longer tested on it.
// A window of fewer than T pixels is one leaf; with `words` it is pixelized from parity words
// (xor_rows) when both polygons are resident, otherwise as row strips against every edge.
// Returns the warp-wide count (the same in every lane). Whole warp, converged.
template <bool TWO, bool COUNT, int CAP, int STK, bool UNION = false>
__device__ __forceinline__ uint32_t pixelbox(const PolyPair pp, int wx0, int wy0, int wx1, int wy1, int T, int words,
                                             WarpSmem<CAP, STK>& S, int lane, WorkCounters& wc)
{
    const int W = wx1 - wx0, H = wy1 - wy0;
    const int fl0 = TWO ? 3 : 1;
    uint32_t acc = 0;
    int top = 0;
    if (COUNT && lane == 0) wc.window_pixels += (unsigned long long)W * H;
    if (words && (long long)W * H < T && pp.rp_res && (!TWO || pp.rq_res)) {
        // The whole window is one leaf: pixelize it from the parity words (xor_rows), in pieces of
        // up to 992 columns and passes of up to 64 rows, one lane per row in the reduction.
        for (int cx = 0; cx < W; cx += 32 * kXorMaxWords) {
            const int Wp = min(32 * kXorMaxWords, W - cx), nw = (Wp + 31) >> 5;
            const int nr = min(64, kXorWords / nw);
            for (int r0 = 0; r0 < H; r0 += nr) {
                const int nrr = min(nr, H - r0);
                for (int k = lane; k < nrr; k += 32) {
                    S.xp.F[k] = 0;
                    if (TWO) S.xq.F[k] = 0;
                }
                for (int k = lane; k < nrr * nw; k += 32) {
                    S.xp.P[k] = 0;
                    if (TWO) S.xq.P[k] = 0;
                }
                __syncwarp();
                unsigned long long ce = 0;
                xor_rows<COUNT>(S.ep, S.rp, pp.np, wx0 + cx, wy0 + r0, nrr, Wp, nw, S.xp, lane, ce);
                if (TWO) xor_rows<COUNT>(S.eq, S.rq, pp.nq, wx0 + cx, wy0 + r0, nrr, Wp, nw, S.xq, lane, ce);
                __syncwarp();
                for (int k = lane; k < nrr; k += 32) {
                    for (int j = 0; j < nw; ++j) {
                        uint32_t in = __funnelshift_lc(0xffffffffu, 0u, (unsigned)min(32, Wp - 32 * j));
                        const uint32_t wp = xor_word(S.xp, k, nw, j) ^ flip_of<CAP>(pp.fp, r0 + k, 0);
                        if (TWO) {
                            const uint32_t wq = xor_word(S.xq, k, nw, j) ^ flip_of<CAP>(pp.fq, r0 + k, 0);
                            in &= UNION ? (wp | wq) : (wp & wq);
                        } else {
                            in &= wp;
                        }
                        acc += __popc(in);
                    }
                    if (COUNT) {
                        wc.row_edges += (unsigned long long)nw;
                        wc.leaf_pixels += (unsigned long long)Wp * (TWO ? 2 : 1);
                    }
                }
                if (COUNT) wc.row_entries += ce;
                __syncwarp();
            }
        }
    } else if ((long long)W * H < T) {
        acc += pixelize_leaves<TWO, COUNT, CAP, STK, UNION>(pp, S, wx0, wy0, lane, pack_box(0, 0, W, H, fl0),
                                                            lane == 0, wc);
    } else {
        if (lane == 0) S.stack[0] = pack_box(0, 0, W, H, fl0);
        top = 1;
    }
    __syncwarp();
    while (top > 0) {
        --top;
        int x0, y0, x1, y1, fl;
        unpack_box(S.stack[top], x0, y0, x1, y1, fl);
        __syncwarp();
        const int w = x1 - x0, h = y1 - y0;
        int gx, gy;
        choose_split(w, h, gx, gy);
        const int nsub = gx * gy;
        const bool mine = lane < nsub;
        const int ix = lane % gx, iy = lane / gx;
        const int sx0 = x0 + (ix * w) / gx, sx1 = x0 + ((ix + 1) * w) / gx;
        const int sy0 = y0 + (iy * h) / gy, sy1 = y0 + ((iy + 1) * h) / gy;
        const int ax0 = wx0 + sx0, ay0 = wy0 + sy0, ax1 = wx0 + sx1, ay1 = wy0 + sy1;
        // 0 outside, 1 inside, 2 hover; a polygon the box no longer needs is inside it for the
        // intersection and outside it for the union
        int posP = UNION ? 0 : 1, posQ = UNION ? 0 : 1;
        unsigned long long ce = 0;
        if (fl & 1) {
            posP = poly_box<COUNT>(pp.vp, pp.np, pp.rp_res, S.ep, S.rp, CAP, ax0, ay0, ax1, ay1,
                                   flip_of<CAP>(pp.fp, ay0, wy0), lane, ce);
            if (COUNT && mine) wc.boxes += 1;
        }
        if (TWO && (fl & 2)) {
            posQ = poly_box<COUNT>(pp.vq, pp.nq, pp.rq_res, S.eq, S.rq, CAP, ax0, ay0, ax1, ay1,
                                   flip_of<CAP>(pp.fq, ay0, wy0), lane, ce);
            if (COUNT && mine) wc.boxes += 1;
        }
        if (COUNT && mine) wc.box_edges += ce;
        const bool out = mine && (UNION ? (posP == 0 && posQ == 0) : (posP == 0 || posQ == 0));
        const bool allin = mine && !out && (UNION ? (posP == 1 || posQ == 1) : (posP == 1 && posQ == 1));
        const int size = (sx1 - sx0) * (sy1 - sy0);
        if (allin) acc += (uint32_t)size;
        const bool cont = mine && !out && !allin;
        const int nfl = (posP == 2 ? 1 : 0) | (posQ == 2 ? 2 : 0);
        // a box that cannot be split further (one sub-box) is pixelized, so the loop always ends
        bool push = cont && size >= T && nsub > 1;
        const unsigned pm = __ballot_sync(kFull, push);
        const int npush = __popc(pm);
        const bool room = top + npush <= STK;
        if (!room) push = false;     // stack full: pixelize instead (still exact)
        const bool leaf = cont && !push;
        if (push) S.stack[top + __popc(pm & ((1u << lane) - 1u))] = pack_box(sx0, sy0, sx1, sy1, nfl);
        if (room) top += npush;
        __syncwarp();
        const bool anyleaf = __any_sync(kFull, leaf);
        if (anyleaf)
            acc += pixelize_leaves<TWO, COUNT, CAP, STK, UNION>(pp, S, wx0, wy0, lane,
                                                                pack_box(sx0, sy0, sx1, sy1, nfl), leaf, wc);
    }
    return warp_sum(acc);
}

}  // namespace sccg
