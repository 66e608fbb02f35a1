// Pixel rasters kept resident with a polygon set, and pair areas from them.
//
// The raster of polygon i is its window of W x H pixels (MBR [x0, x1) x [y0, y1)) as H rows of
// nw = ceil(W / 32) words: bit b of word k of row r is set iff pixel (x0 + 32 k + b, y0 + r) belongs
// to the polygon under the pixel-centre ray-casting rule of Sec. 3.1. Buffer layout: int64 off[n + 1]
// (polygon i's first word; off[n] the total) padded to 16 bytes, then the words: a slot of
// kRasterSlot words for every polygon (polygon i's at kRasterSlot * i, used when its window is at
// most 64 x 64 pixels, so that k_prepare writes it in the same pass that finds the MBR), then the
// rasters of the larger windows, placed once k_prepare has listed them.
//
// Every (pixel, polygon) membership is then decided once per polygon, when the set is prepared,
// instead of once for every pair the polygon takes part in: ||p n q|| of a pair is the popcount of
// the AND of the two rasters' rows over the overlap of their MBRs (a4), and ||p u q|| follows from
// the areas as before (a5). The rasters of windows up to 64 x 64 pixels are the leaf parity rows of
// k_prepare; larger ones are drawn here (k_raster_big) from difference rows.
//
// Difference rows. An edge that straddles row y crosses the first c pixels of the row right of x0
// (c = crossing_count_r, Sec. 3.1 in doubled coordinates), so pixel x0 + t belongs to the polygon iff
// an odd number of the row's crossings have c > t. Each crossing toggles bit c of a row of bits D;
// pixel t is then the XOR of D's bits above t (an exclusive suffix XOR along the row). A pass covers
// up to 32 PIECE columns (a piece starting at column cs) of a group of rows: a crossing
// with c <= cs changes no pixel of the piece and is dropped, one with c beyond the piece toggles the
// piece's overflow bit (position 32 nwp, after the piece's nwp words), which flips the whole piece.
#pragma once
#include <cstdint>

#include "kernels.cuh"

namespace sccg {

// Per-warp difference words: 32 rows of a piece of PIECE words plus the overflow word. Polygons drawn
// from their rings take pieces of 32 words (1024 columns: a small buffer, many resident warps);
// polygons with band lists, whose passes are one 32-row band each, take 64 (2048 columns: each
// band's list read half as often).
template <int PIECE>
struct DrawSmem {
    uint32_t D[32 * (PIECE + 1)];
};

__host__ __device__ inline long long raster_head_bytes(long long n)
{
    return (8 * (n + 1) + 15) & ~15LL;
}


// Toggle the difference bits of the crossings of one group of edges (lane k holds edge
// {ylo, dy, dx, xl}, lower endpoint first, when `has`) with window rows ya .. ya + nr - 1 (absolute
// y), piece columns cs .. cs + 32 nwp - 1 of a window whose left column is x0. Row q of the pass is
// D[q * (nwp + 1) ...]. When no edge of the group spans more than kLeafLoopSpan of the rows, each
// lane walks its own edge's rows; otherwise the (edge, row) crossings are spread evenly over the
// lanes (warp prefix sum of the edges' row counts, owner found by binary search, edge fetched by
// shuffles). Whole warp, converged; the trip counts are warp-uniform.
__device__ __forceinline__ void draw_group(bool has, int ylo, int dy, int dx, int xl, int x0, int ya, int nr, int cs,
                                           int nwp, uint32_t* D, int lane, unsigned long long& entries)
{
    int cnt = 0;
    if (has && max(xl, xl + dx) > x0 + cs) cnt = max(0, min(ylo + dy, ya + nr) - max(ylo, ya));
    const int maxc = __reduce_max_sync(kFull, cnt);
    if (maxc == 0) return;
    const float r2 = cnt > 0 ? __frcp_rn((float)(2 * dy)) : 0.0f;     // dy > 0 whenever cnt > 0
    const int stride = nwp + 1, pmax = 32 * nwp;
    if (maxc <= kLeafLoopSpan) {
        // short spans: each lane walks its own edge's rows
        const int y0e = max(ylo, ya);
#pragma unroll
        for (int s = 0; s < kLeafLoopSpan; ++s) {
            if (s >= maxc) break;
            if (s < cnt) {
                const int y = y0e + s;
                const int p = min(crossing_count_r(ylo, dy, dx, xl, y, x0, r2) - cs, pmax);
                if (p > 0) atomicXor(&D[(y - ya) * stride + (p >> 5)], 1u << (p & 31));
            }
        }
        entries += (unsigned long long)cnt;
        return;
    }
    int total;
    const int excl = warp_excl(cnt, lane, total);
    for (int t0 = 0; t0 < total; t0 += 32) {
        const int t = t0 + lane;
        const int own = flat_owner(excl, t);
        const int eo = __shfl_sync(kFull, excl, own);
        const int oy = __shfl_sync(kFull, ylo, own), ody = __shfl_sync(kFull, dy, own);
        const int odx = __shfl_sync(kFull, dx, own), oxl = __shfl_sync(kFull, xl, own);
        const float orr = __shfl_sync(kFull, r2, own);
        if (t < total) {
            const int y = max(oy, ya) + (t - eo);
            const int p = min(crossing_count_r(oy, ody, odx, oxl, y, x0, orr) - cs, pmax);
            if (p > 0) atomicXor(&D[(y - ya) * stride + (p >> 5)], 1u << (p & 31));
        }
    }
    entries += (unsigned long long)cnt;
}

// All crossings of the edges of `src` (RingEdges or RecordEdges) with one pass. Whole warp.
template <class Edges>
__device__ __forceinline__ void draw_pass(const Edges src, int x0, int ya, int nr, int cs, int nwp, uint32_t* D,
                                          int lane, unsigned long long& entries)
{
    for (int base = 0; base < src.n; base += 32) {
        const int e = base + lane;
        int ylo = 0, dy = 0, dx = 0, xl = 0;
        if (e < src.n) src.get(e, ylo, dy, dx, xl);
        draw_group(e < src.n, ylo, dy, dx, xl, x0, ya, nr, cs, nwp, D, lane, entries);
    }
}

// The raster words of one pass from its difference rows: row q of the pass goes to out + q * nw
// (words cs / 32 ..), one lane per row, words taken right to left with the parity of every toggle
// to their right. Returns this lane's count of member pixels. Columns at or beyond W are cleared.
__device__ __forceinline__ uint32_t draw_finish(const uint32_t* D, int nr, int nwp, int cs, int W, int nw,
                                                uint32_t* out, int lane)
{
    uint32_t acc = 0;
    const int stride = nwp + 1, k0 = cs >> 5;
    for (int q = lane; q < nr; q += 32) {
        const uint32_t* d = D + q * stride;
        uint32_t par = __popc(d[nwp]) & 1u;            // toggles beyond the piece flip all of it
        for (int j = nwp - 1; j >= 0; --j) {
            const uint32_t w = d[j];
            uint32_t x = w;                              // bit t: XOR of bits t .. 31 of w
            x ^= x >> 1;
            x ^= x >> 2;
            x ^= x >> 4;
            x ^= x >> 8;
            x ^= x >> 16;
            uint32_t bits = (x >> 1) ^ (par ? 0xffffffffu : 0u);
            const int col = cs + 32 * j;
            if (W - col < 32) bits &= low_mask(W - col);
            par ^= __popc(w) & 1u;
            out[(long long)q * nw + k0 + j] = bits;
            acc += __popc(bits);
        }
    }
    return acc;
}

// The next list position from a counter, for the whole warp. Whole warp, converged.
__device__ __forceinline__ long long claim_next(unsigned* next, int lane)
{
    unsigned t = 0;
    if (lane == 0) t = atomicAdd(next, 1u);
    return (long long)__shfl_sync(kFull, t, 0);
}

// Rasters and ||p|| of the polygons k_prepare listed (windows over 64 pixels wide or high): pieces of
// up to 32 PIECE columns, passes of as many rows as the per-warp difference words hold. Otherwise
// (BANDED false) only the polygons without a block in the band index blob, one warp each, streaming
// the whole ring once per pass; BANDED: only the polygons with a block (large tissue regions), one
// CTA each, its warps taking the 32-row bands in turn, each band's edges from the band's list, and
// the warps' counts summed in shared memory. next (BANDED false; zero at the launch): the list
// position the next free warp takes, so that warps drawing small windows take more of them.
template <bool COUNT, int PIECE, bool BANDED>
__global__ void __launch_bounds__(256) k_raster_big(const int64_t* off, const int32_t* xy, const int4* mbr,
                                                    const char* blob, const int* list, const unsigned* n_list,
                                                    int64_t* area, const long long* roff, uint32_t* rwords,
                                                    WorkCounters* counters, unsigned* next)
{
    constexpr int kWords = 32 * (PIECE + 1);
    SCCG_DYNAMIC_SMEM(int4, smem4);
    __shared__ unsigned part[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, wpb = blockDim.x >> 5;
    DrawSmem<PIECE>& S = reinterpret_cast<DrawSmem<PIECE>*>(smem4)[warp];
    WorkCounters wc = {};
    const long long nl = *n_list;
    const long long step = BANDED ? gridDim.x : (long long)gridDim.x * wpb;
    unsigned* const dyn = BANDED ? nullptr : next;
    const long long first = dyn ? claim_next(dyn, lane) : BANDED ? blockIdx.x : (long long)blockIdx.x * wpb + warp;
    for (long long j = first; j < nl; j = dyn ? claim_next(dyn, lane) : j + step) {
        const long long i = list[j];
        const char* blk = band_block(blob, i);
        if ((blk != nullptr) != BANDED) continue;                // uniform per warp (per CTA when BANDED)
        const long long o0 = off[i];
        const int nv = (int)(off[i + 1] - o0);
        const int2* v = reinterpret_cast<const int2*>(xy) + o0;
        const int4 m = mbr[i];
        const int W = m.z - m.x, H = m.w - m.y, nw = (W + 31) >> 5;
        uint32_t* out = rwords + roff[i];
        uint32_t acc = 0;
        unsigned long long ce = 0;
        for (int cs = 0; cs < W; cs += 32 * PIECE) {
            const int nwp = min(PIECE, nw - (cs >> 5));
            // band lists cover 32 rows each (from the polygon's min y): one band per pass
            const int nrmax = BANDED ? (1 << kBandShift) : kWords / (nwp + 1);
            for (int r0 = BANDED ? warp * nrmax : 0; r0 < H; r0 += BANDED ? wpb * nrmax : nrmax) {
                const int nr = min(nrmax, H - r0);
                __syncwarp();
                for (int k = lane; k < nr * (nwp + 1); k += 32) S.D[k] = 0u;
                __syncwarp();
                if (BANDED) {
                    const int nb = reinterpret_cast<const int*>(blk)[0];
                    const int* boff = reinterpret_cast<const int*>(blk) + 4;
                    const int4* ent = reinterpret_cast<const int4*>(blk + 16 + ((4LL * (2 * nb + 1) + 15) & ~15LL));
                    const int b = r0 >> kBandShift;
                    if (b < nb)
                        draw_pass(RecordEdges{ent + boff[b], boff[b + 1] - boff[b]}, m.x, m.y + r0, nr, cs, nwp,
                                  S.D, lane, ce);
                } else {
                    draw_pass(RingEdges{v, nv}, m.x, m.y + r0, nr, cs, nwp, S.D, lane, ce);
                }
                __syncwarp();
                acc += draw_finish(S.D, nr, nwp, cs, W, nw, out + (long long)r0 * nw, lane);
            }
        }
        acc = warp_sum(acc);
        if (BANDED) {
            if (lane == 0) part[warp] = acc;
            __syncthreads();
            if (threadIdx.x == 0) {
                unsigned long long t = 0;
                for (int w = 0; w < wpb; ++w) t += part[w];
                area[i] = (int64_t)t;
            }
            __syncthreads();
        } else if (lane == 0) {
            area[i] = (int64_t)acc;
        }
        if (COUNT) {
            wc.scan_entries += ce;
            if (lane == 0 && (!BANDED || warp == 0)) {
                wc.raster_out += (unsigned long long)raster_words_of(W, H);
                wc.window_pixels += (unsigned long long)W * H;
            }
        }
    }
    if (COUNT) flush_counters(counters, wc);
}

// Word counts of the rasters of the polygons k_prepare listed (windows over 64 pixels wide or high).
__global__ void k_raster_sizes(const int* list, const unsigned* n_list, const int4* mbr, long long* words)
{
    const long long nl = *n_list;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nl; j += (long long)gridDim.x * blockDim.x) {
        const int4 m = mbr[list[j]];
        words[j] = raster_words_of(m.z - m.x, m.w - m.y);
    }
}

// Header entries of the listed polygons, placed after the n leaf slots in list order (offs: the
// exclusive scan of their word counts, offs[nl] their total), and rhead[n] = the rasters' total words.
__global__ void k_raster_place(const int* list, const unsigned* n_list, const long long* offs, long long n,
                               long long* rhead)
{
    const long long nl = *n_list;
    const long long base = (long long)kRasterSlot * n;
    for (long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x; j < nl; j += (long long)gridDim.x * blockDim.x)
        rhead[list[j]] = base + offs[j];
    if (blockIdx.x == 0 && threadIdx.x == 0) rhead[n] = base + offs[nl];
}

// ----------------------------------------------------------------------------------------------
// a4 + a5 from rasters
// ----------------------------------------------------------------------------------------------
struct RasterPairArgs {
    long long n;
    long long nA, nB;
    const int32_t* pa;
    const int32_t* pb;
    const int4* mbrA; const int64_t* areaA; const long long* roffA; const uint32_t* rwA;
    const int4* mbrB; const int64_t* areaB; const long long* roffB; const uint32_t* rwB;
    int64_t* inter;
    int64_t* uni;
    long long heavy_words;          // pairs with more (row, word) units are listed for the CTA kernel
                                    // (< 0: every pair is done by its warp)
    unsigned long long* heavy;      // the list (pair indices)
    unsigned long long* heavy_n;    // its length
    unsigned long long* head;       // chunk counter (nullptr: static grid-stride over chunks)
    WorkCounters* counters;
};

// One pair's window in both rasters: word index of the overlap's first row in each, words per row,
// bit offset of the overlap's first column, and the overlap's size.
struct RPair {
    long long pA, pB;
    int nwa, nwb, sa, sb, W, H;
};

__device__ __forceinline__ RPair raster_window(const int4 ma, const int4 mb, long long offa, long long offb)
{
    RPair t;
    const int ox0 = max(ma.x, mb.x), oy0 = max(ma.y, mb.y);
    t.W = max(min(ma.z, mb.z) - ox0, 0);
    t.H = max(min(ma.w, mb.w) - oy0, 0);
    if (t.W == 0) t.H = 0;
    t.nwa = (ma.z - ma.x + 31) >> 5;
    t.nwb = (mb.z - mb.x + 31) >> 5;
    t.sa = ox0 - ma.x;
    t.sb = ox0 - mb.x;
    t.pA = offa + (long long)(oy0 - ma.y) * t.nwa;
    t.pB = offb + (long long)(oy0 - mb.y) * t.nwb;
    return t;
}

// Member pixels of both polygons in word q (columns 32 q .. 32 q + 31 of the overlap) of the rows
// ra, rb (each row's word 0 is the raster's first word of that row).
__device__ __forceinline__ uint32_t raster_and_word(const uint32_t* ra, const uint32_t* rb, const RPair& t, int q)
{
    const int s = t.sa + 32 * q, u = t.sb + 32 * q;
    const int ka = s >> 5, kb = u >> 5;
    const uint32_t a0 = ra[ka], a1 = ka + 1 < t.nwa ? ra[ka + 1] : 0u;
    const uint32_t b0 = rb[kb], b1 = kb + 1 < t.nwb ? rb[kb + 1] : 0u;
    uint32_t w = __funnelshift_r(a0, a1, (unsigned)s & 31u) & __funnelshift_r(b0, b1, (unsigned)u & 31u);
    const int left = t.W - 32 * q;
    if (left < 32) w &= low_mask(left);
    return (uint32_t)__popc(w);
}

// Light pairs: each warp takes 32 consecutive pairs (a chunk); lane j reads pair j's MBRs, raster
// offsets and areas into a shared table, then the warp goes through the chunk's pairs G lanes per
// pair (32 / G pairs at a time, so that their row loads are in flight together), lanes over the
// overlap's rows, and writes the 32 results together. G = 1: each lane does its own pair when the
// window is at most 64 x 64 pixels, row after row, and the warp the others. Heavy pairs (more than
// heavy_words (row, word) units) are listed for k_pair_raster_heavy. A pair whose indices are out of
// range gets -1.
template <bool COUNT, int G>
__global__ void __launch_bounds__(256) k_pair_raster(const RasterPairArgs a)
{
    __shared__ RPair tab[8][32];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    WorkCounters wc = {};
    const long long stride = (long long)gridDim.x * (blockDim.x >> 5) * 32;
    long long base = ((long long)blockIdx.x * (blockDim.x >> 5) + warp) * 32;
    for (;;) {
        if (a.head) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(a.head, 32ull);
            base = (long long)__shfl_sync(kFull, b, 0);
        }
        if (base >= a.n) break;
        const long long k = base + lane;
        bool valid = false, light = false, own = false;
        long long sum_area = 0;
        RPair t = {};
        if (k < a.n) {
            const int ia = a.pa[k], ib = a.pb[k];
            if (ia >= 0 && ia < a.nA && ib >= 0 && ib < a.nB) {
                valid = true;
                t = raster_window(a.mbrA[ia], a.mbrB[ib], a.roffA[ia], a.roffB[ib]);
                const long long units = (long long)t.H * ((t.W + 31) >> 5);
                light = a.heavy_words < 0 || units <= a.heavy_words;
                own = G == 1 && light && t.W <= kLeafSide && t.H <= kLeafSide;
                sum_area = a.areaA[ia] + a.areaB[ib];
                tab[warp][lane] = t;
                if (!light) a.heavy[atomicAdd(a.heavy_n, 1ull)] = (unsigned long long)k;
                else if (t.H > 0) {
                    // the window's rows of both rasters (contiguous, the first 1 KB of each) requested into
                    // L2 now: the chunk's pairs are ANDed one group after another below
                    const char* ra = reinterpret_cast<const char*>(a.rwA + t.pA);
                    const char* rb = reinterpret_cast<const char*>(a.rwB + t.pB);
                    const int na = min(4 * t.H * t.nwa, 1024), nb = min(4 * t.H * t.nwb, 1024);
                    for (int o = 0; o < na; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(ra + o));
                    for (int o = 0; o < nb; o += 128) asm volatile("prefetch.global.L2 [%0];" ::"l"(rb + o));
                }
            }
        }
        __syncwarp();
        uint32_t mine = 0;
        if (G == 1 && own && t.H > 0) {
            // one lane per pair whose window is at most 64 x 64 pixels: its rows one after another
            const int nwo = (t.W + 31) >> 5;
            const uint32_t* ra = a.rwA + t.pA;
            const uint32_t* rb = a.rwB + t.pB;
#pragma unroll 4
            for (int r = 0; r < t.H; ++r)
                for (int q = 0; q < nwo; ++q)
                    mine += raster_and_word(ra + (long long)r * t.nwa, rb + (long long)r * t.nwb, t, q);
            if (COUNT) {
                wc.raster_and += (unsigned long long)t.H * nwo;
                wc.window_pixels += (unsigned long long)t.W * t.H;
            }
        }
        unsigned todo = __ballot_sync(kFull, light && !own && tab[warp][lane].H > 0);
        // GW lanes per pair: the warp takes 32 / GW of the chunk's pairs at a time, one per lane group
        // (with G = 1, the pairs no lane took alone go to the whole warp)
        constexpr int GW = G == 1 ? 32 : G;
        const int grp = lane / GW, gl = lane % GW;
        const unsigned gmask = GW == 32 ? kFull : (((1u << GW) - 1u) << (grp * GW));
        while (todo) {
            int my = -1;
#pragma unroll
            for (int g = 0; g < 32 / GW; ++g) {
                if (todo) {
                    const int j = __ffs(todo) - 1;
                    todo &= todo - 1;
                    if (g == grp) my = j;
                }
            }
            uint32_t acc = 0;
            if (my >= 0) {
                const RPair u = tab[warp][my];
                const int nwo = (u.W + 31) >> 5;
                for (int r = gl; r < u.H; r += GW) {
                    const uint32_t* ra = a.rwA + u.pA + (long long)r * u.nwa;
                    const uint32_t* rb = a.rwB + u.pB + (long long)r * u.nwb;
                    for (int q = 0; q < nwo; ++q) acc += raster_and_word(ra, rb, u, q);
                }
                if (COUNT && gl == 0) {
                    wc.raster_and += (unsigned long long)u.H * nwo;
                    wc.window_pixels += (unsigned long long)u.W * u.H;
                }
            }
            const uint32_t tot = __reduce_add_sync(gmask, acc);
#pragma unroll
            for (int g = 0; g < 32 / GW; ++g) {
                const uint32_t tg = __shfl_sync(kFull, tot, g * GW);
                const int jg = __shfl_sync(kFull, my, g * GW);
                if (lane == jg) mine = tg;
            }
        }
        if (k < a.n && (light || !valid)) {
            a.inter[k] = valid ? (int64_t)mine : -1;
            a.uni[k] = valid ? sum_area - (int64_t)mine : -1;
        }
        __syncwarp();
        if (!a.head) base += stride;
    }
    if (COUNT) flush_counters(a.counters, wc);
}

// Heavy pairs, one CTA per pair (grid-stride over the list): the 8 warps take rows in turn; within a
// warp, lanes cover the overlap's words, several rows at once when a row has fewer than 32 words.
template <bool COUNT>
__global__ void __launch_bounds__(256) k_pair_raster_heavy(const RasterPairArgs a)
{
    __shared__ uint32_t part[8];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
    WorkCounters wc = {};
    const unsigned long long nh = *a.heavy_n;
    for (unsigned long long h = blockIdx.x; h < nh; h += gridDim.x) {
        const long long k = (long long)a.heavy[h];
        const int ia = a.pa[k], ib = a.pb[k];
        const RPair t = raster_window(a.mbrA[ia], a.mbrB[ib], a.roffA[ia], a.roffB[ib]);
        const int nwo = (t.W + 31) >> 5;
        // lane -> (row within the warp's group, first word); rows per group: 32 / nwo when nwo < 32
        const int sub = nwo < 32 ? 32 / nwo : 1;
        const int lr = nwo < 32 ? lane / nwo : 0;
        const int q0 = nwo < 32 ? lane - lr * nwo : lane;
        const int qstep = nwo < 32 ? nwo : 32;
        uint32_t acc = 0;
        if (lr < sub) {
            for (int r = warp * sub + lr; r < t.H; r += nwarp * sub) {
                const uint32_t* ra = a.rwA + t.pA + (long long)r * t.nwa;
                const uint32_t* rb = a.rwB + t.pB + (long long)r * t.nwb;
                for (int q = q0; q < nwo; q += qstep) acc += raster_and_word(ra, rb, t, q);
            }
        }
        acc = __reduce_add_sync(kFull, acc);
        if (lane == 0) part[warp] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t s = 0;
            for (int w = 0; w < nwarp; ++w) s += part[w];
            a.inter[k] = (int64_t)s;
            a.uni[k] = a.areaA[ia] + a.areaB[ib] - (int64_t)s;
            if (COUNT) {
                wc.raster_and += (unsigned long long)t.H * nwo;
                wc.window_pixels += (unsigned long long)t.W * t.H;
            }
        }
        __syncthreads();
    }
    if (COUNT) flush_counters(a.counters, wc);
}

}  // namespace sccg
