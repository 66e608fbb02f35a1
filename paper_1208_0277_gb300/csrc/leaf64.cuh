// Leaf windows of at most 64 x 64 pixels (Sec. 3.1 ray casting on a box below the threshold T,
// Sec. 3.2), pixelized edge-major from per-row parity words, for one polygon or both polygons of a
// pair at once.
//
// An edge that straddles pixel row y crosses exactly the first c pixels of the row right of the
// window's left column x0 (the rule of pixelbox.cuh: pixel x0 + t is crossed iff 2 t dy < N with
// N = (2 (y - ylo) + 1) dx - (2 (x0 - xl) + 1) dy), so it flips the parity of those c pixels. Each
// polygon keeps one 64-bit parity word per row (two 32-bit halves in shared memory); an edge's
// crossing XORs the prefix mask of its c pixels into its row, and a pixel's final bit is its ray's
// crossing parity: set iff the pixel is inside the polygon.
//
// The edges of both rings are streamed through registers as one sequence (lane k of a batch holds
// edge k of P, or edge k - n_P of Q), so a nucleus pair of ~70 edges takes three batches of 32. An
// edge spans few rows of a small window, so each lane walks its own edge's rows (trip count = the
// warp's longest span); only a batch holding an edge that spans more than kLeafLoopSpan rows spreads
// its (edge, row) crossings evenly over the lanes (prefix sum and owner search, as xor_group).
#pragma once
#include <cstdint>

#include "pixelbox.cuh"

namespace sccg {

constexpr int kLeafSide = 64;             // largest window side handled here
constexpr int kLeafQ = 144;               // first word of Q's rows: 16 banks after P's
constexpr int kLeafWords = kLeafQ + 128;  // P: rows 0..63 of pixels 0..31, then of pixels 32..63; Q alike
constexpr int kLeafLoopSpan = 3;          // longest edge span (rows) walked lane by lane

// Per-warp parity words. Word base + 64 h + r holds pixels 32 h .. 32 h + 31 of window row r of the
// polygon whose rows start at `base` (0 for P, kLeafQ for Q).
struct Leaf64 {
    uint32_t w[kLeafWords];
};

// Low min(c, 32) bits set (c >= 0).
__device__ __forceinline__ uint32_t low_mask(int c)
{
    return __funnelshift_lc(0xffffffffu, 0u, (unsigned)c);
}

// Approximate reciprocal (PTX rcp.approx.ftz.f32: at most one ulp from 1/x, relative error at most
// 2^-23).
__device__ __forceinline__ float rcp_approx(float x)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Exact int -> float for 0 <= v < 2^23 (the integer placed in the significand of 2^23).
__device__ __forceinline__ float small_int_to_float(int v)
{
    return __int_as_float(v | 0x4B000000) - 8388608.0f;
}

// c = ceil(D / d2) for 0 <= D <= 64 d2, d2 = 2 dy with 1 <= dy <= 2^14, rc = rcp_approx(d2).
// D < 2^22 converts exactly. fma(D, rc, -2^-16) is x - 2^-16 (x = D / d2 <= 64) up to the
// reciprocal's error (x * 2^-23 <= 2^-17) and the fma's one rounding (<= 64 * 2^-24 = 2^-18), so it
// lies in [x - 3.5 * 2^-17, x - 0.5 * 2^-17]. An integer x thus gives a value in (x - 1, x), and a
// non-integer x, which lies at least 1 / d2 >= 2^-15 = 4 * 2^-17 above the integer m below it, a value
// in (m, x): rounding up gives ceil(D / d2) exactly in both cases. The ceiling is taken by an
// upward-rounded add of 1.5 * 2^23, where floats are spaced one apart.
__device__ __forceinline__ int leaf_ceil_div(int D, float rc)
{
    const float q = __fmaf_rn(small_int_to_float(D), rc, -1.52587890625e-05f);
    return __float_as_int(__fadd_ru(q, 12582912.0f)) - 0x4B400000;
}

// One edge held by a lane, set up against the window [x0, x0 + W) x [y0, y0 + H): it straddles
// `span` rows from window row rlo - y0 on, whose words start at w = base + rlo - y0; at its s-th
// row N = N0 + s * dx2. cap = 64 d2 (N is clamped to [0, cap]: at most 64 crossed pixels matter).
// In the own-window form N0 and dx2 are also held as floats (N0f, dx2f): every N of a window of at
// most 64 x 64 pixels is an integer of magnitude at most 129 * 64 + 129 * 64 < 2^24, so
// fma(s, dx2f, N0f) is N exactly.
struct LeafEdge {
    int N0, dx2, cap, w, span;
    float rc, N0f, dx2f;
};

// The crossing of an edge with a straddled row (N, words w and w + 64): XOR the prefix mask of its
// c = ceil(clamp(N, 0, cap) / d2) crossed pixels into the row's halves (pixels beyond the window's
// width are masked off when the rows are counted). WIDE: the window is over 32 pixels wide. SELF: the
// window is the polygon's own MBR, so no edge crosses beyond its width (N <= W d2 <= cap) and the upper
// clamp is not needed.
template <bool WIDE, bool SELF = false>
__device__ __forceinline__ void leaf_cross(int N, int cap, float rc, int w, Leaf64& L)
{
    const int c = leaf_ceil_div(SELF ? max(N, 0) : min(max(N, 0), cap), rc);
    const uint32_t lo = low_mask(c);
    if (lo) atomicXor(&L.w[w], lo);
    if (WIDE) {
        const uint32_t hi = low_mask(max(c - 32, 0));
        if (hi) atomicXor(&L.w[w + 64], hi);
    }
}

// leaf_cross of the own-window form with N held exactly as a float (LeafEdge): the clamp at 0 and
// the quotient of leaf_ceil_div on the float directly.
template <bool WIDE>
__device__ __forceinline__ void leaf_cross_f(float N, float rc, int w, Leaf64& L)
{
    const float q = __fmaf_rn(fmaxf(N, 0.0f), rc, -1.52587890625e-05f);
    const int c = __float_as_int(__fadd_ru(q, 12582912.0f)) - 0x4B400000;
    const uint32_t lo = low_mask(c);
    if (lo) atomicXor(&L.w[w], lo);
    if (WIDE) {
        const uint32_t hi = low_mask(max(c - 32, 0));
        if (hi) atomicXor(&L.w[w + 64], hi);
    }
}

// All crossings of the batch's edges (one per lane, set up in e; maxs = the warp's longest span)
// with the window's rows. Spans of at most kLeafLoopSpan rows: each lane walks its own edge's rows.
// Longer ones: the batch's (edge, row) crossings are spread evenly over the lanes (warp prefix sum of
// the spans; each lane finds its crossing's edge by a binary search over the lanes' offsets and
// fetches it by shuffles). Whole warp, converged.
template <bool COUNT, bool WIDE, bool SELF = false>
__device__ __forceinline__ void leaf_batch_w(const LeafEdge& e, int maxs, Leaf64& L, int lane,
                                             unsigned long long& entries)
{
    if (COUNT) entries += (unsigned long long)e.span;
    if (maxs <= kLeafLoopSpan) {
#pragma unroll
        for (int s = 0; s < kLeafLoopSpan; ++s) {
            if (s >= maxs) break;
            if (s < e.span) {
                if (SELF) leaf_cross_f<WIDE>(__fmaf_rn((float)s, e.dx2f, e.N0f), e.rc, e.w + s, L);
                else leaf_cross<WIDE>(e.N0 + s * e.dx2, e.cap, e.rc, e.w + s, L);
            }
        }
        return;
    }
    int total;
    const int excl = warp_excl(e.span, lane, total);
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        const int own = flat_owner(excl, t);
        const int s = t - __shfl_sync(kFull, excl, own);
        const int w = __shfl_sync(kFull, e.w, own);
        const float rc = __shfl_sync(kFull, e.rc, own);
        if (SELF) {
            const float N0f = __shfl_sync(kFull, e.N0f, own);
            const float dx2f = __shfl_sync(kFull, e.dx2f, own);
            if (t < total) leaf_cross_f<WIDE>(__fmaf_rn(small_int_to_float(max(s, 0)), dx2f, N0f), rc, w + s, L);
        } else {
            const int N0 = __shfl_sync(kFull, e.N0, own);
            const int dx2 = __shfl_sync(kFull, e.dx2, own);
            const int cap = __shfl_sync(kFull, e.cap, own);
            if (t < total) leaf_cross<WIDE>(N0 + s * dx2, cap, rc, w + s, L);
        }
    }
}

// One batch of edges, lane k holding edge a -> b (either order; `has` false past the ring's end) of
// the polygon whose rows start at word `base`, against the window [x0, x0 + W) x [y0, y0 + H).
// The rows an edge straddles are found first, and a batch with none stops there. An edge with no
// point right of x0 crosses no pixel centre of the window (every centre lies right of x = x0), and a
// horizontal one straddles no row: both get span 0. Every product is below 2^30 under the library's
// coordinate and extent limits (|N| <= (2 dy) |dx| + (2 |x0 - xl| + 1) dy with dy, |dx|, |x0 - xl|
// at most 2^14 + 64). SELF: the window is the polygon's own MBR, so every edge lies inside it: its rows
// from ylo to yhi are all window rows, and an edge on the left border crosses no pixel (its c is 0).
// Whole warp, converged.
template <bool COUNT, bool SELF = false>
__device__ __forceinline__ void leaf_batch(bool has, int2 a, int2 b, int x0, int y0, int W, int H, int base,
                                           Leaf64& L, int lane, unsigned long long& entries)
{
    const bool up = a.y <= b.y;
    const int ylo = up ? a.y : b.y, yhi = up ? b.y : a.y;
    const int rlo = SELF ? ylo : max(ylo, y0);
    LeafEdge e;
    e.span = SELF ? (has ? yhi - ylo : 0) : (has && max(a.x, b.x) > x0) ? max(min(yhi, y0 + H) - rlo, 0) : 0;
    const int maxs = __reduce_max_sync(kFull, e.span);
    if (maxs == 0) return;
    const int xl = up ? a.x : b.x;
    const int dy = yhi - ylo, dx = (up ? b.x : a.x) - xl;
    const int d2 = dy + dy;
    e.dx2 = dx + dx;
    e.N0 = SELF ? dx - (2 * (x0 - xl) + 1) * dy : (2 * (rlo - ylo) + 1) * dx - (2 * (x0 - xl) + 1) * dy;
    e.cap = d2 << 6;
    e.rc = rcp_approx(small_int_to_float(max(d2, 1)));
    if (SELF) {
        e.N0f = __int2float_rn(e.N0);
        e.dx2f = __int2float_rn(e.dx2);
    }
    e.w = base + rlo - y0;
    if (W > 32) leaf_batch_w<COUNT, true, SELF>(e, maxs, L, lane, entries);
    else leaf_batch_w<COUNT, false, SELF>(e, maxs, L, lane, entries);
}

// The edges of ring vp[0 .. np) (rows at word basep) followed by those of ring vq[0 .. nq) (rows at
// baseq; nq may be 0), 32 at a time. Whole warp, converged; the trip count is warp-uniform.
template <bool COUNT, bool SELF = false>
__device__ __forceinline__ void leaf_rings(const int2* vp, int np, int basep, const int2* vq, int nq, int baseq,
                                           int x0, int y0, int W, int H, Leaf64& L, int lane,
                                           unsigned long long& entries)
{
    const int E = np + nq;
    for (int b0 = 0; b0 < E; b0 += 32) {
        const int k = b0 + lane;
        const bool has = k < E;
        const bool isq = k >= np;
        const int kk = isq ? k - np : k;
        const int n = isq ? nq : np;
        const int2* v = isq ? vq : vp;
        int2 a = make_int2(0, 0), b = make_int2(0, 0);
        if (has) {
            a = v[kk];
            b = v[kk + 1 == n ? 0 : kk + 1];
        }
        leaf_batch<COUNT, SELF>(has, a, b, x0, y0, W, H, isq ? baseq : basep, L, lane, entries);
    }
}

// Zero the rows of the window (P's, and Q's when two). Whole warp.
__device__ __forceinline__ void leaf_clear(Leaf64& L, int W, int H, bool two, int lane)
{
    for (int r = lane; r < H; r += 32) {
        L.w[r] = 0u;
        if (W > 32) L.w[64 + r] = 0u;
        if (two) {
            L.w[kLeafQ + r] = 0u;
            if (W > 32) L.w[kLeafQ + 64 + r] = 0u;
        }
    }
}

// Pixels of the window inside P (and inside Q when two), summed over the warp (every lane gets it).
template <bool COUNT>
__device__ __forceinline__ uint32_t leaf_pixels(const Leaf64& L, int W, int H, bool two, int lane, WorkCounters& wc)
{
    const uint32_t vlo = low_mask(W), vhi = low_mask(max(W - 32, 0));
    uint32_t acc = 0;
    for (int r = lane; r < H; r += 32) {
        uint32_t lo = L.w[r] & vlo;
        if (two) lo &= L.w[kLeafQ + r];
        acc += __popc(lo);
        if (W > 32) {
            uint32_t hi = L.w[64 + r] & vhi;
            if (two) hi &= L.w[kLeafQ + 64 + r];
            acc += __popc(hi);
        }
        if (COUNT) {
            wc.row_edges += W > 32 ? 2ull : 1ull;
            wc.leaf_pixels += (unsigned long long)W * (two ? 2 : 1);
        }
    }
    return __reduce_add_sync(kFull, acc);
}

// ||p|| of a polygon whose bounding box [x0, x1) x [y0, y1) is at most 64 x 64 pixels, as one leaf:
// its ring streamed once. With out, the rows are also written there as the polygon's raster (H rows
// of one or two words), in the pass that counts them, and cleared in that pass: the caller zeroes
// P's rows once before its first call with out, and they are zero again after every call. Whole
// warp, converged.
template <bool COUNT>
__device__ __forceinline__ uint32_t leaf_area(const int2* v, int nv, int x0, int y0, int x1, int y1, Leaf64& L,
                                              int lane, WorkCounters& wc, uint32_t* out = nullptr)
{
    const int W = x1 - x0, H = y1 - y0;
    if (COUNT && lane == 0) wc.window_pixels += (unsigned long long)W * H;
    if (!out) {
        __syncwarp();
        leaf_clear(L, W, H, false, lane);
    }
    __syncwarp();
    unsigned long long ce = 0;
    leaf_rings<COUNT, true>(v, nv, 0, v, 0, 0, x0, y0, W, H, L, lane, ce);
    __syncwarp();
    uint32_t a;
    if (out) {
        const uint32_t vlo = low_mask(W), vhi = low_mask(max(W - 32, 0));
        uint32_t acc = 0;
        for (int r = lane; r < H; r += 32) {
            const uint32_t lo = L.w[r] & vlo;
            L.w[r] = 0u;
            if (W > 32) {
                const uint32_t hi = L.w[64 + r] & vhi;
                L.w[64 + r] = 0u;
                out[2 * r] = lo;
                out[2 * r + 1] = hi;
                acc += __popc(lo) + __popc(hi);
            } else {
                out[r] = lo;
                acc += __popc(lo);
            }
            if (COUNT) {
                wc.row_edges += W > 32 ? 2ull : 1ull;
                wc.leaf_pixels += (unsigned long long)W;
            }
        }
        a = __reduce_add_sync(kFull, acc);
        if (COUNT && lane == 0) wc.raster_out += (unsigned long long)H * (W > 32 ? 2 : 1);
    } else {
        a = leaf_pixels<COUNT>(L, W, H, false, lane, wc);
    }
    if (COUNT) wc.row_entries += ce;
    __syncwarp();
    return a;
}

}  // namespace sccg
