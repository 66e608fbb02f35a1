// C ABI of the cross-comparison library (declared in include/sccg.h): argument validation, scratch
// management and kernel launches. Every step of the path runs in the kernels of kernels.cuh.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>

#include "kernels.cuh"
#include "raster.cuh"
#include "sccg.h"

using namespace sccg;

namespace {

constexpr int kStack = 160;         // sampling-box stack entries per warp
constexpr uint32_t kPreparedMagic = 0x5CC6A11u;

}  // namespace

struct sccg_ctx {
    int device = 0;
    int sm_count = 0;
    sccg_params params{};
    void* ws = nullptr;             // device scratch
    size_t ws_size = 0;
    // separately growable scratch: candidate-pair grid cells, cell entries, prepare's temporary band
    // index, the candidate pairs' per-polygon B lists
    void* aux[4] = {nullptr, nullptr, nullptr, nullptr};
    size_t aux_size[4] = {0, 0, 0, 0};
    void* pinned = nullptr;         // small host-pinned staging area
    void* pinned_dev = nullptr;     // ... as addressed by kernels
    WorkCounters* counters = nullptr;   // device work counters (counting mode)
    int count_work = 0;
    // candidate pairs: grid buffers sized before the counts are known (1), only from the counts
    // (0, two more synchronisations), or too small on purpose (2, to test the redo); per B polygon
    int cand_speculative = 1;
    double cand_cells_per_b = 2.0;
    double cand_entries_per_b = 4.0;
    unsigned long long launches = 0;    // kernels launched by this context (all calls)
    static constexpr int kTileStreams = 8;
    cudaStream_t tstream[kTileStreams] = {};
    cudaEvent_t tevent[kTileStreams + 1] = {};
    bool tile_streams_ready = false;
    // second stream of the persistent form (the big-polygon queue runs beside the small one)
    cudaStream_t side_stream = nullptr;
    cudaEvent_t fork_event = nullptr, join_event = nullptr;
    // sccg_batch_run: the captured graph and the arguments it was captured for
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t batch_exec = nullptr;
    const void* batch_key[13] = {};
    long long batch_n = -1;
    sccg_params batch_params{};
    int batch_count_work = 0;
    unsigned long long batch_launches = 0;   // kernels launched by one replay of the graph
    char last_err[256] = {0};
};

namespace {

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_fail(sccg_ctx* ctx, cudaError_t e, const char* where)
{
    if (ctx) snprintf(ctx->last_err, sizeof ctx->last_err, "%s: %s", where, cudaGetErrorString(e));
    return SCCG_ECUDA;
}

#define SCCG_CUDA(ctx, call)                                          \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call);    \
    } while (0)

#define SCCG_LAUNCHED(ctx, what)                                      \
    do {                                                              \
        cudaError_t e_ = cudaGetLastError();                          \
        if (e_ != cudaSuccess) return cuda_fail((ctx), e_, what);     \
    } while (0)

bool is_device_ptr(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Grow the device scratch to at least `bytes` (synchronises the device when it grows).
int ws_reserve(sccg_ctx* ctx, size_t bytes)
{
    if (bytes <= ctx->ws_size) return SCCG_OK;
    size_t want = std::max(bytes, ctx->ws_size * 3 / 2);
    want = (want + 0xFFFFF) & ~size_t(0xFFFFF);
    if (ctx->ws) {
        cudaDeviceSynchronize();
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_size = 0;
    }
    if (cudaMalloc(&ctx->ws, want) != cudaSuccess) {
        cudaGetLastError();
        snprintf(ctx->last_err, sizeof ctx->last_err, "scratch allocation of %zu bytes failed", want);
        return SCCG_ENOMEM;
    }
    ctx->ws_size = want;
    return SCCG_OK;
}

// Grow auxiliary scratch buffer k to at least `bytes` (its previous contents are not kept).
int aux_reserve(sccg_ctx* ctx, int k, size_t bytes)
{
    if (bytes <= ctx->aux_size[k]) return SCCG_OK;
    size_t want = std::max(bytes, ctx->aux_size[k] * 3 / 2);
    want = (want + 0xFFFFF) & ~size_t(0xFFFFF);
    if (ctx->aux[k]) {
        cudaDeviceSynchronize();
        cudaFree(ctx->aux[k]);
        ctx->aux[k] = nullptr;
        ctx->aux_size[k] = 0;
    }
    if (cudaMalloc(&ctx->aux[k], want) != cudaSuccess) {
        cudaGetLastError();
        snprintf(ctx->last_err, sizeof ctx->last_err, "scratch allocation of %zu bytes failed", want);
        return SCCG_ENOMEM;
    }
    ctx->aux_size[k] = want;
    return SCCG_OK;
}

// Bump allocator over the scratch (256-byte aligned pieces).
struct Carve {
    char* base;
    size_t used = 0;
    explicit Carve(void* b) : base(static_cast<char*>(b)) {}
    template <class T>
    T* take(size_t count)
    {
        used = (used + 255) & ~size_t(255);
        T* p = reinterpret_cast<T*>(base + used);
        used += count * sizeof(T);
        return p;
    }
};
template <class T>
size_t carve_size(size_t count) { return ((count * sizeof(T) + 255) & ~size_t(255)) + 256; }

#ifndef SCCG_CAP_MID
#define SCCG_CAP_MID 128
#endif
constexpr int kCopyCTAs = 16;      // CTAs of sccg_copy: 16 x 512 threads fill the host link (~211 GB/s)
constexpr int kMaxPrepSets = 64;  // sets per sccg_prepare_sets call (their stats share the pinned page)
static_assert(kMaxPrepSets * sizeof(PrepStats) <= 4096, "prepare stats must fit the pinned staging page");
constexpr int kCapSmall = 64;     // edge buffer of the one-warp-per-item kernels (4 warps per CTA)
constexpr int kCapMid = SCCG_CAP_MID;   // persistent form, pairs with a polygon over kCapSmall vertices
constexpr int kCapBig = 512;      // edge buffer for polygons with more vertices (2 warps per CTA)
#ifndef SCCG_CAP_OVF
#define SCCG_CAP_OVF 256
#endif
#ifndef SCCG_WARPS_256
#define SCCG_WARPS_256 2
#endif
#ifndef SCCG_STREAM
#define SCCG_STREAM 1     // persistent form: stream the edges when every item is one leaf
#endif
#ifndef SCCG_LEAF
#define SCCG_LEAF 1       // ... through k_pair_areas_leaf when items are at most 64 x 64 pixels
#endif
// persistent form: first overflow level (0: items over kCapMid go straight to kCapBig)
constexpr int kCapOvf = SCCG_CAP_OVF;
static_assert(kCapOvf == 0 || (kCapOvf > kCapMid && kCapOvf < kCapBig), "overflow levels must grow");

int edge_cap_for(int max_nv) { return max_nv <= kCapSmall ? kCapSmall : kCapBig; }
int warps_for(const sccg_ctx* ctx, int cap)
{
    const int w = std::max(1, std::min(8, ctx->params.warps_per_cta));
    return cap >= kCapBig ? std::min(w, 2) : cap > kCapMid ? std::min(w, SCCG_WARPS_256) : w;
}

template <int CAP>
size_t warp_smem() { return sizeof(WarpSmem<CAP, kStack>); }

template <class K>
int set_smem(sccg_ctx* ctx, K kernel, size_t bytes)
{
    if (bytes > 48 * 1024)
        SCCG_CUDA(ctx, cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
    return SCCG_OK;
}

long long grid_for(const sccg_ctx* ctx, long long items, int per_block, int max_blocks_per_sm)
{
    long long g = (items + per_block - 1) / per_block;
    const long long cap = (long long)ctx->sm_count * max_blocks_per_sm;
    if (g > cap) g = cap;
    if (g < 1) g = 1;
    return g;
}

// Zero `bytes` (a multiple of 4) of device memory, and copy `bytes` (a multiple of 8, 8-byte
// aligned, at most a few KB) between device memory and the pinned staging area, by kernels: the
// copy engines may be busy with a caller's bulk copies of the next batch.
int zero_async(sccg_ctx* ctx, void* p, size_t bytes, cudaStream_t st)
{
    const long long n = (long long)(bytes / 4);
    if (n <= 0) return SCCG_OK;
    const long long g = std::min<long long>((n + 255) / 256, 4LL * ctx->sm_count);
    k_zero32<<<(unsigned)g, 256, 0, st>>>(static_cast<uint32_t*>(p), n);
    SCCG_LAUNCHED(ctx, "k_zero32");
    ctx->launches += 1;
    return SCCG_OK;
}

int small_copy(sccg_ctx* ctx, void* dst, const void* src, size_t bytes, cudaStream_t st)
{
    k_copy64<<<1, 128, 0, st>>>(static_cast<const unsigned long long*>(src), static_cast<unsigned long long*>(dst),
                                (int)(bytes / 8));
    SCCG_LAUNCHED(ctx, "k_copy64");
    ctx->launches += 1;
    return SCCG_OK;
}

template <class K>
int persistent_grid(sccg_ctx* ctx, K kfn, int wpc, size_t smem, unsigned* grid)
{
    int per_sm = ctx->params.ctas_per_sm;
    if (per_sm <= 0) {
        SCCG_CUDA(ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kfn, 32 * wpc, smem));
        per_sm = std::max(per_sm, 1);
    }
    *grid = (unsigned)(ctx->sm_count * per_sm);
    return SCCG_OK;
}

template <int PIECE, bool BANDED>
int launch_raster_big(sccg_ctx* ctx, const sccg_polyset* s, const char* blob, const int* list, const unsigned* n_list,
                      unsigned n_host, const long long* rhead, uint32_t* rw, const int4* mbr, unsigned* next,
                      cudaStream_t st)
{
    const int wpc = BANDED ? 8 : 4;          // BANDED: one CTA per polygon, its warps taking bands in turn
    const size_t smem = sizeof(DrawSmem<PIECE>) * wpc;
    auto kfn = ctx->count_work ? k_raster_big<true, PIECE, BANDED> : k_raster_big<false, PIECE, BANDED>;
    int r = set_smem(ctx, kfn, smem);
    unsigned resident = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &resident);
    if (r) return r;
    // at most the resident CTAs: each warp then draws polygon after polygon (a CTA holding one polygon
    // per warp would keep its slot until its largest polygon is done)
    const unsigned grid = std::max(1u, std::min(BANDED ? n_host : (n_host + wpc - 1) / wpc, resident));
    kfn<<<grid, 32 * wpc, smem, st>>>(s->off, s->xy, mbr, blob, list, n_list, s->area, rhead, rw, ctx->counters,
                                      BANDED ? nullptr : next);
    SCCG_LAUNCHED(ctx, "k_raster_big");
    ctx->launches += 1;
    return SCCG_OK;
}

int launch_mbr(sccg_ctx* ctx, const PrepArgs& a, long long* words, cudaStream_t st)
{
    const long long grid = grid_for(ctx, a.n, 8, 8);     // the resident CTAs, one polygon per warp in turn
    k_mbr<<<(unsigned)grid, 256, 0, st>>>(a, words);
    SCCG_LAUNCHED(ctx, "k_mbr");
    ctx->launches += 1;
    return SCCG_OK;
}

template <int CAP, bool SCAN, bool RASTER = false>
int launch_prepare(sccg_ctx* ctx, const PrepArgs& a, cudaStream_t st)
{
    const int wpc = warps_for(ctx, CAP);
    const size_t smem = (SCAN ? kPrepWarpBytes : warp_smem<CAP>()) * wpc;    // SCAN: streamed leaves only
    const long long grid = grid_for(ctx, a.n, wpc, 64);
    auto kfn = ctx->count_work ? k_prepare<CAP, kStack, true, SCAN, RASTER> : k_prepare<CAP, kStack, false, SCAN, RASTER>;
    int r = set_smem(ctx, kfn, smem);
    if (r) return r;
    kfn<<<(unsigned)grid, 32 * wpc, smem, st>>>(a);
    SCCG_LAUNCHED(ctx, "k_prepare");
    ctx->launches += 1;
    return SCCG_OK;
}

template <int CAP>
int launch_prepare_big(sccg_ctx* ctx, const PrepArgs& a, cudaStream_t st)
{
    const int wpc = warps_for(ctx, CAP);
    const size_t smem = warp_smem<CAP>() * wpc;
    auto kfn = ctx->count_work ? k_prepare_big<CAP, kStack, true> : k_prepare_big<CAP, kStack, false>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);     // every warp slot of the device
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a);
    SCCG_LAUNCHED(ctx, "k_prepare_big");
    ctx->launches += 1;
    return SCCG_OK;
}

int raster_launch(sccg_ctx* ctx, const AreasArgs& a, bool persistent, cudaStream_t st);

template <int CAP, bool NOSEP = false>
int launch_plain(sccg_ctx* ctx, const AreasArgs& a, cudaStream_t st)
{
    if (!NOSEP && a.rwA && a.rwB) return raster_launch(ctx, a, false, st);
    const int wpc = warps_for(ctx, CAP);
    const size_t smem = warp_smem<CAP>() * wpc;
    const long long grid = grid_for(ctx, a.n, wpc, 64);
    auto kfn = NOSEP ? (ctx->count_work ? k_pair_areas_nosep<CAP, kStack, true> : k_pair_areas_nosep<CAP, kStack, false>)
                     : (ctx->count_work ? k_pair_areas_plain<CAP, kStack, true> : k_pair_areas_plain<CAP, kStack, false>);
    int r = set_smem(ctx, kfn, smem);
    if (r) return r;
    kfn<<<(unsigned)grid, 32 * wpc, smem, st>>>(a);
    SCCG_LAUNCHED(ctx, NOSEP ? "k_pair_areas_nosep" : "k_pair_areas_plain");
    ctx->launches += 1;
    return SCCG_OK;
}

template <int CAP, bool OVF>
int launch_persistent(sccg_ctx* ctx, const AreasArgs& a, int side, const long long* nitems, const long long* ioff,
                      unsigned long long* head, unsigned long long* ovf_list, unsigned long long* ovf_n,
                      long long ovf_cap, cudaStream_t st)
{
    const int wpc = warps_for(ctx, CAP);
    const size_t smem = warp_smem<CAP>() * wpc;
    auto kfn = ctx->count_work ? k_pair_areas_persistent<CAP, kStack, true, OVF>
                               : k_pair_areas_persistent<CAP, kStack, false, OVF>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a, side, nitems, ioff, head, ovf_list, ovf_n, ovf_cap);
    SCCG_LAUNCHED(ctx, "k_pair_areas_persistent");
    ctx->launches += 1;
    return SCCG_OK;
}

int launch_stream(sccg_ctx* ctx, const AreasArgs& a, int side, const long long* nitems, const long long* ioff,
                  unsigned long long* head, cudaStream_t st)
{
    const int wpc = warps_for(ctx, kCapSmall);
    const size_t smem = sizeof(StreamSmem) * wpc;
    auto kfn = ctx->count_work ? k_pair_areas_stream<true> : k_pair_areas_stream<false>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a, side, nitems, ioff, head);
    SCCG_LAUNCHED(ctx, "k_pair_areas_stream");
    ctx->launches += 1;
    return SCCG_OK;
}

int launch_lanes(sccg_ctx* ctx, const AreasArgs& a, const long long* lane, cudaStream_t st)
{
    constexpr int wpc = 2;                               // k_pair_areas_lanes: CTAs of 64 threads
    const size_t smem = sizeof(LaneSmem) * wpc;
    auto kfn = ctx->count_work ? k_pair_areas_lanes<true> : k_pair_areas_lanes<false>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a, lane);
    SCCG_LAUNCHED(ctx, "k_pair_areas_lanes");
    ctx->launches += 1;
    return SCCG_OK;
}

int launch_leaf(sccg_ctx* ctx, const AreasArgs& a, int side, const long long* ioff, unsigned long long* head,
                cudaStream_t st)
{
    const int wpc = warps_for(ctx, kCapSmall);
    const size_t smem = sizeof(LeafSmem) * wpc;
    auto kfn = ctx->count_work ? k_pair_areas_leaf<true> : k_pair_areas_leaf<false>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a, side, ioff, head);
    SCCG_LAUNCHED(ctx, "k_pair_areas_leaf");
    ctx->launches += 1;
    return SCCG_OK;
}

template <int CAP, bool OVF>
int launch_overflow(sccg_ctx* ctx, const AreasArgs& a, int side, const long long* nitems,
                    const unsigned long long* ovf_list, const unsigned long long* ovf_n, long long ovf_cap,
                    unsigned long long* head, unsigned long long* ovf2_list, unsigned long long* ovf2_n,
                    long long ovf2_cap, cudaStream_t st)
{
    const int wpc = warps_for(ctx, CAP);
    const size_t smem = warp_smem<CAP>() * wpc;
    auto kfn = ctx->count_work ? k_pair_areas_overflow<CAP, kStack, true, OVF>
                               : k_pair_areas_overflow<CAP, kStack, false, OVF>;
    int r = set_smem(ctx, kfn, smem);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, wpc, smem, &grid);
    if (r) return r;
    kfn<<<grid, 32 * wpc, smem, st>>>(a, side, nitems, ovf_list, ovf_n, ovf_cap, head, ovf2_list, ovf2_n, ovf2_cap);
    SCCG_LAUNCHED(ctx, "k_pair_areas_overflow");
    ctx->launches += 1;
    return SCCG_OK;
}

int check_prepared(const sccg_polyset* s)
{
    if (!s) return SCCG_EINVAL;
    if ((uint32_t)s->reserved != kPreparedMagic) return SCCG_EINVAL;
    if (s->n < 0 || s->n > 0x7fffffffLL) return SCCG_EINVAL;
    return SCCG_OK;
}

// Point the pair-area arguments at both sets' rasters when both have them and the context uses them.
void use_rasters(const sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, AreasArgs& a)
{
    if (!ctx->params.rasters || !A->raster_ok || !B->raster_ok || !A->raster || !B->raster) return;
    a.roffA = static_cast<const long long*>(A->raster);
    a.rwA = reinterpret_cast<const uint32_t*>(static_cast<const char*>(A->raster) + raster_head_bytes(A->n));
    a.roffB = static_cast<const long long*>(B->raster);
    a.rwB = reinterpret_cast<const uint32_t*>(static_cast<const char*>(B->raster) + raster_head_bytes(B->n));
}

// exclusive scan of counts[n] into offs[n+1]; scratch from carve
int device_scan(sccg_ctx* ctx, const long long* counts, long long n, long long* offs, long long* bsum,
                cudaStream_t st)
{
    if (n == 0) {
        return zero_async(ctx, offs, sizeof(long long), st);
    }
    const long long nb = (n + kScanBlock - 1) / kScanBlock;
    k_scan_reduce<<<(unsigned)nb, kScanBlock, 0, st>>>(counts, n, bsum);
    k_scan_top<<<1, kScanBlock, 0, st>>>(bsum, nb);
    k_scan_apply<<<(unsigned)nb, kScanBlock, 0, st>>>(counts, n, bsum, offs);
    SCCG_LAUNCHED(ctx, "device_scan");
    ctx->launches += 3;
    return SCCG_OK;
}

// overflow list capacity of the persistent form (items beyond it are done in place, chunked)
long long overflow_cap(long long n_pairs) { return n_pairs + 65536; }
// ... of the second level (items that do not fit the first overflow level's buffers either)
long long overflow2_cap(long long n_pairs) { return kCapOvf ? n_pairs / 4 + 65536 : 0; }

size_t persistent_scratch(long long n_pairs)
{
    const long long nb = (n_pairs + kScanBlock - 1) / kScanBlock + 1;
    return carve_size<long long>(n_pairs + 1) * 4 + carve_size<long long>(nb) + carve_size<unsigned long long>(4) +
           carve_size<long long>(overflow_cap(n_pairs)) + carve_size<long long>(overflow2_cap(n_pairs));
}

int split_side(const sccg_ctx* ctx)
{
    int side = 1;
    while ((long long)(side + 1) * (side + 1) <= ctx->params.split_pixels) ++side;
    return side;
}

// Pair areas from both sets' rasters. persistent: chunks of 32 pairs taken from a device counter
// by resident CTAs, heavy pairs listed and done one CTA each (scratch from the persistent form's
// reservation); otherwise a static grid-stride with every pair done by its warp.
int raster_launch(sccg_ctx* ctx, const AreasArgs& a, bool persistent, cudaStream_t st)
{
    RasterPairArgs ra{a.n, a.nA, a.nB, a.pa, a.pb,
                      a.mbrA, a.areaA, a.roffA, a.rwA, a.mbrB, a.areaB, a.roffB, a.rwB,
                      a.inter, a.uni, -1, nullptr, nullptr, nullptr, a.counters};
    const int G = ctx->params.raster_lanes;
    auto kfn = ctx->count_work ? (G == 1 ? k_pair_raster<true, 1> : G == 8 ? k_pair_raster<true, 8>
                                  : G == 16 ? k_pair_raster<true, 16> : k_pair_raster<true, 32>)
                               : (G == 1 ? k_pair_raster<false, 1> : G == 8 ? k_pair_raster<false, 8>
                                  : G == 16 ? k_pair_raster<false, 16> : k_pair_raster<false, 32>);
    if (!persistent) {
        const long long grid = grid_for(ctx, (a.n + 31) / 32, 8, 16);
        kfn<<<(unsigned)grid, 256, 0, st>>>(ra);
        SCCG_LAUNCHED(ctx, "k_pair_raster");
        ctx->launches += 1;
        return SCCG_OK;
    }
    Carve cv(ctx->ws);
    unsigned long long* cnt = cv.take<unsigned long long>(2);       // chunk head, heavy count
    ra.heavy = cv.take<unsigned long long>(a.n);
    ra.head = cnt;
    ra.heavy_n = cnt + 1;
    ra.heavy_words = ctx->params.raster_heavy;
    int r = zero_async(ctx, cnt, 2 * sizeof(unsigned long long), st);
    unsigned grid = 0;
    if (!r) r = persistent_grid(ctx, kfn, 8, 0, &grid);
    if (r) return r;
    kfn<<<grid, 256, 0, st>>>(ra);
    SCCG_LAUNCHED(ctx, "k_pair_raster");
    ctx->launches += 1;
    if (ra.heavy_words >= 0) {
        auto hfn = ctx->count_work ? k_pair_raster_heavy<true> : k_pair_raster_heavy<false>;
        r = persistent_grid(ctx, hfn, 8, 0, &grid);
        if (r) return r;
        hfn<<<grid, 256, 0, st>>>(ra);
        SCCG_LAUNCHED(ctx, "k_pair_raster_heavy");
        ctx->launches += 1;
    }
    return SCCG_OK;
}

// Persistent form on already reserved scratch (no validation, no allocation: usable under capture).
int persistent_launch(sccg_ctx* ctx, const AreasArgs& a, int cap, cudaStream_t st)
{
    if (a.rwA && a.rwB) return raster_launch(ctx, a, true, st);
    const long long n_pairs = a.n;
    const int side = split_side(ctx);
    const long long nb = (n_pairs + kScanBlock - 1) / kScanBlock + 1;
    Carve cv(ctx->ws);
    long long* nitems_s = cv.take<long long>(n_pairs + 1);
    long long* nitems_b = cv.take<long long>(n_pairs + 1);
    long long* ioff_s = cv.take<long long>(n_pairs + 1);
    long long* ioff_b = cv.take<long long>(n_pairs + 1);
    long long* bsum = cv.take<long long>(nb);
    // queue heads: small, big, overflow 1, overflow 2; counts: overflow 1, overflow 2
    unsigned long long* head = cv.take<unsigned long long>(6);
    const long long ovf_cap = overflow_cap(n_pairs);
    unsigned long long* ovf_list = cv.take<unsigned long long>(ovf_cap);
    const long long ovf2_cap = overflow2_cap(n_pairs);
    unsigned long long* ovf2_list = cv.take<unsigned long long>(ovf2_cap);
    const unsigned g = (unsigned)((n_pairs + 255) / 256);
    if (SCCG_LEAF && ctx->params.leaf_words && side <= kLeafSide && (long long)side * side < ctx->params.T) {
        // every item is one leaf of at most 64 x 64 pixels: the items through the leaf kernel's queue;
        // with pair_lanes = 1 small pairs one lane each, on the side stream beside it
        const bool lanes = ctx->params.pair_lanes == 1;
        k_plan_leaf<<<g, 256, 0, st>>>(a, side, lanes ? 1 : 0, nitems_s, nitems_b);
        SCCG_LAUNCHED(ctx, "k_plan_leaf");
        ctx->launches += 1;
        int r = device_scan(ctx, nitems_s, n_pairs, ioff_s, bsum, st);
        if (!r) r = zero_async(ctx, head, sizeof(unsigned long long), st);
        if (r) return r;
        if (lanes) {
            SCCG_CUDA(ctx, cudaEventRecord(ctx->fork_event, st));
            SCCG_CUDA(ctx, cudaStreamWaitEvent(ctx->side_stream, ctx->fork_event, 0));
            r = launch_lanes(ctx, a, nitems_b, ctx->side_stream);
            if (r) return r;
            SCCG_CUDA(ctx, cudaEventRecord(ctx->join_event, ctx->side_stream));
        }
        r = launch_leaf(ctx, a, side, ioff_s, head, st);
        if (r) return r;
        if (lanes) SCCG_CUDA(ctx, cudaStreamWaitEvent(st, ctx->join_event, 0));
        k_union<<<g, 256, 0, st>>>(a, nitems_s, nitems_b);
        SCCG_LAUNCHED(ctx, "k_union");
        ctx->launches += 1;
        return SCCG_OK;
    }
    if (SCCG_STREAM && ctx->params.leaf_words && (long long)side * side < ctx->params.T) {
        // every item is one leaf: one queue, edges streamed from the rings (no edge buffers)
        k_plan<<<g, 256, 0, st>>>(a, side, 0x7fffffff, nitems_s, nitems_b);
        SCCG_LAUNCHED(ctx, "k_plan");
        ctx->launches += 1;
        int r = device_scan(ctx, nitems_s, n_pairs, ioff_s, bsum, st);
        if (!r) r = zero_async(ctx, head, sizeof(unsigned long long), st);
        if (!r) r = launch_stream(ctx, a, side, nitems_s, ioff_s, head, st);
        if (r) return r;
        k_union<<<g, 256, 0, st>>>(a, nitems_s, nitems_b);
        SCCG_LAUNCHED(ctx, "k_union");
        ctx->launches += 1;
        return SCCG_OK;
    }
    // pairs whose polygons all fit the small edge buffers go to one queue, the rest to another
    k_plan<<<g, 256, 0, st>>>(a, side, kCapSmall, nitems_s, nitems_b);
    SCCG_LAUNCHED(ctx, "k_plan");
    ctx->launches += 1;
    int r = device_scan(ctx, nitems_s, n_pairs, ioff_s, bsum, st);
    if (!r && cap > kCapSmall) r = device_scan(ctx, nitems_b, n_pairs, ioff_b, bsum, st);
    if (r) return r;
    r = zero_async(ctx, head, 6 * sizeof(unsigned long long), st);
    if (r) return r;
    if (cap > kCapSmall) {
        // the big-polygon queue on the side stream, beside the small one: mid-size buffers, and the
        // items whose culled edges still do not fit go to the largest buffers afterwards
        SCCG_CUDA(ctx, cudaEventRecord(ctx->fork_event, st));
        SCCG_CUDA(ctx, cudaStreamWaitEvent(ctx->side_stream, ctx->fork_event, 0));
        r = launch_persistent<kCapMid, true>(ctx, a, side, nitems_b, ioff_b, head + 1, ovf_list, head + 4, ovf_cap,
                                             ctx->side_stream);
        if (kCapOvf) {
            // two overflow levels: kCapOvf-edge buffers, then the largest for what still does not fit
            if (!r) r = launch_overflow<kCapOvf ? kCapOvf : kCapBig, true>(ctx, a, side, nitems_b, ovf_list, head + 4,
                                                                           ovf_cap, head + 2, ovf2_list, head + 5,
                                                                           ovf2_cap, ctx->side_stream);
            if (!r) r = launch_overflow<kCapBig, false>(ctx, a, side, nitems_b, ovf2_list, head + 5, ovf2_cap, head + 3,
                                                        nullptr, nullptr, 0, ctx->side_stream);
        } else if (!r) {
            r = launch_overflow<kCapBig, false>(ctx, a, side, nitems_b, ovf_list, head + 4, ovf_cap, head + 2, nullptr,
                                                nullptr, 0, ctx->side_stream);
        }
        if (r) return r;
        SCCG_CUDA(ctx, cudaEventRecord(ctx->join_event, ctx->side_stream));
    }
    r = launch_persistent<kCapSmall, false>(ctx, a, side, nitems_s, ioff_s, head, nullptr, nullptr, 0, st);
    if (r) return r;
    if (cap > kCapSmall) SCCG_CUDA(ctx, cudaStreamWaitEvent(st, ctx->join_event, 0));
    k_union<<<g, 256, 0, st>>>(a, nitems_s, nitems_b);
    SCCG_LAUNCHED(ctx, "k_union");
    ctx->launches += 1;
    return SCCG_OK;
}

int jaccard_parts(const sccg_ctx* ctx, long long n_pairs)
{
    return (int)std::max(1LL, std::min<long long>((n_pairs + 255) / 256, 4LL * ctx->sm_count));
}

size_t jaccard_scratch(const sccg_ctx* ctx, long long n_pairs)
{
    return carve_size<JPart>(jaccard_parts(ctx, n_pairs)) + carve_size<JaccardOut>(1);
}

// Jaccard into a device result on already reserved scratch (no validation, no allocation).
int jaccard_launch(sccg_ctx* ctx, const int64_t* inter, const int64_t* uni, long long n_pairs, JaccardOut* res,
                   cudaStream_t st)
{
    const int nparts = jaccard_parts(ctx, n_pairs);
    Carve cv(ctx->ws);
    JPart* parts = cv.take<JPart>(nparts);
    k_jaccard_partial<<<nparts, 256, 0, st>>>(inter, uni, n_pairs, parts);
    k_jaccard_final<<<1, 256, 0, st>>>(parts, nparts, n_pairs, res);
    SCCG_LAUNCHED(ctx, "k_jaccard");
    ctx->launches += 2;
    return SCCG_OK;
}

// Band index of set s into blob (at least band_bytes(s) bytes), scratch from `cv`. Asynchronous.
int build_bands_into(sccg_ctx* ctx, const sccg_polyset* s, char* blob, long long bytes, Carve& cv, cudaStream_t st)
{
    const long long n = s->n;
    const long long nb = (n + kScanBlock - 1) / kScanBlock + 1;
    long long* size = cv.take<long long>(n + 1);
    long long* boffs = cv.take<long long>(n + 1);
    long long* bsum = cv.take<long long>(nb);
    const int4* mbr = reinterpret_cast<const int4*>(s->mbr);
    const unsigned gw = (unsigned)grid_for(ctx, n, 8, 16);      // 8 warps per CTA, one polygon per warp
    k_band_sizes<<<gw, 256, 0, st>>>(n, s->off, s->xy, mbr, size);
    SCCG_LAUNCHED(ctx, "k_band_sizes");
    const int r = device_scan(ctx, size, n, boffs, bsum, st);
    if (r) return r;
    k_band_tab<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(n, size, boffs, blob, bytes);
    SCCG_LAUNCHED(ctx, "k_band_tab");
    k_band_fill<<<gw, 256, 0, st>>>(n, s->off, s->xy, mbr, blob);
    SCCG_LAUNCHED(ctx, "k_band_fill");
    ctx->launches += 3;
    return SCCG_OK;
}

size_t band_build_scratch(long long n)
{
    return carve_size<long long>(n + 1) * 2 + carve_size<long long>((n + kScanBlock - 1) / kScanBlock + 1);
}

int parse_params(const char* js, sccg_params* p)
{
    if (!js) return SCCG_OK;
    static const char* names[] = {"T", "warps_per_cta", "split_pixels", "ctas_per_sm", "area_method", "leaf_words",
                                  "pair_lanes", "area_T", "rasters", "raster_heavy", "raster_lanes"};
    int32_t* fields[] = {&p->T, &p->warps_per_cta, &p->split_pixels, &p->ctas_per_sm, &p->area_method,
                         &p->leaf_words, &p->pair_lanes, &p->area_T, &p->rasters, &p->raster_heavy, &p->raster_lanes};
    for (int k = 0; k < 11; ++k) {
        char key[64];
        snprintf(key, sizeof key, "\"%s\"", names[k]);
        const char* at = strstr(js, key);
        if (!at) continue;
        at = strchr(at + strlen(key), ':');
        if (!at) return SCCG_EINVAL;
        char* end = nullptr;
        const long v = strtol(at + 1, &end, 10);
        if (end == at + 1) return SCCG_EINVAL;
        *fields[k] = (int32_t)v;
    }
    return SCCG_OK;
}

int validate_params(const sccg_params& p)
{
    if (p.T < 2 || p.T > (1 << 28)) return SCCG_EINVAL;
    if (p.warps_per_cta < 1 || p.warps_per_cta > 8) return SCCG_EINVAL;
    if (p.split_pixels < 32) return SCCG_EINVAL;
    if (p.ctas_per_sm < 0 || p.ctas_per_sm > 64) return SCCG_EINVAL;
    if (p.area_method != SCCG_AREA_ROWS && p.area_method != SCCG_AREA_PIXELBOX && p.area_method != SCCG_AREA_SHOELACE)
        return SCCG_EINVAL;
    if (p.leaf_words != 0 && p.leaf_words != 1) return SCCG_EINVAL;
    if (p.pair_lanes != 1 && p.pair_lanes != 32) return SCCG_EINVAL;
    if (p.area_T < 2 || p.area_T > (1 << 28)) return SCCG_EINVAL;
    if (p.rasters != 0 && p.rasters != 1) return SCCG_EINVAL;
    if (p.raster_heavy < -1) return SCCG_EINVAL;
    if (p.raster_lanes != 1 && p.raster_lanes != 8 && p.raster_lanes != 16 && p.raster_lanes != 32)
        return SCCG_EINVAL;
    return SCCG_OK;
}

// ------------------------------------------------------------------------------------------------
// Allocation-free Jaccard: the partial sums live in a fixed array in device global memory instead
// of context scratch, for callers that may not allocate device memory (see include/sccg.h).
// ------------------------------------------------------------------------------------------------
constexpr int kStaticParts = 4096;            // partial-sum slots in the fixed array
constexpr long long kStaticChunk = 65536;     // pairs reduced into one slot
constexpr long long kStaticMaxPairs = kStaticParts * kStaticChunk;   // 268,435,456 pairs

// One CTA reduces pairs [blockIdx.x * chunk, min(n, (blockIdx.x + 1) * chunk)) into parts[blockIdx.x],
// exactly as k_jaccard_partial does for its grid-stride share.
__global__ void __launch_bounds__(256) k_jaccard_partial_chunked(const int64_t* __restrict__ inter,
                                                                 const int64_t* __restrict__ uni, long long n,
                                                                 long long chunk, JPart* parts)
{
    unsigned long long si = 0, su = 0, nz = 0;
    unsigned __int128 fx = 0;
    const long long lo_i = (long long)blockIdx.x * chunk;
    const long long hi_i = min(n, lo_i + chunk);
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

// The fixed scratch array. Every GPU that loads this library holds it until the process exits.
static __device__ __align__(256) JPart g_jaccard_static_parts[kStaticParts];

// Device address of the fixed array in the current context. It is looked up on every call rather
// than cached: a context created by the caller (cuCtxCreate) holds its own copy of the array, and a
// device reset can load the library's module at another address, so a cached address could belong
// to another context. (The host-side name of a __device__ variable is not a device address and is
// never passed to a kernel.)
int static_parts_address(JPart** out)
{
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_jaccard_static_parts);
    if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return SCCG_ECUDA;
    }
    *out = static_cast<JPart*>(p);
    return SCCG_OK;
}

// p is device (or managed) memory of device `dev`.
// The address by which kernels on device dev reach p: device memory of dev, or page-locked host
// memory mapped into the device's address space; nullptr for anything else (pageable host memory,
// another device's memory, unknown pointers).
void* device_view(const void* p, int dev)
{
    if (!p) return nullptr;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged)
        return at.device == dev ? at.devicePointer : nullptr;
    if (at.type == cudaMemoryTypeHost) return at.devicePointer;
    return nullptr;
}

bool is_device_ptr_on(const void* p, int dev)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) && at.device == dev;
}

}  // namespace

extern "C" {

const char* sccg_status_str(int s)
{
    switch (s) {
        case SCCG_OK: return "ok";
        case SCCG_EINVAL: return "invalid argument";
        case SCCG_ERANGE: return "coordinate or polygon extent out of range";
        case SCCG_ECAPACITY: return "output capacity too small";
        case SCCG_ENOMEM: return "out of device memory";
        case SCCG_ECUDA: return "CUDA error";
        case SCCG_ETIMEOUT: return "device wait timed out";
        case SCCG_ENOTSUP: return "not supported";
        default: return "unknown status";
    }
}

int sccg_ctx_create(int device, const char* params_json, sccg_ctx** out)
{
    if (!out) return SCCG_EINVAL;
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
        cudaGetLastError();
        return ndev == 0 ? SCCG_ENOTSUP : SCCG_EINVAL;
    }
    sccg_ctx* ctx = new (std::nothrow) sccg_ctx();
    if (!ctx) return SCCG_ENOMEM;
    ctx->device = device;
    ctx->params.T = 8192;
    ctx->params.warps_per_cta = 4;
    ctx->params.split_pixels = 4096;
    ctx->params.ctas_per_sm = 0;
    ctx->params.area_method = SCCG_AREA_ROWS;
    ctx->params.leaf_words = 1;
    ctx->params.pair_lanes = 32;
    ctx->params.area_T = 65536;
    ctx->params.rasters = 1;
    ctx->params.raster_heavy = 1024;
    ctx->params.raster_lanes = 32;
    int r = parse_params(params_json, &ctx->params);
    if (!r) r = validate_params(ctx->params);
    if (r) { delete ctx; return r; }
    DeviceGuard g(device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) { delete ctx; return SCCG_ECUDA; }
    ctx->sm_count = prop.multiProcessorCount;
    if (cudaMallocHost(&ctx->pinned, 4096) != cudaSuccess) { cudaGetLastError(); delete ctx; return SCCG_ENOMEM; }
    if (cudaHostGetDevicePointer(&ctx->pinned_dev, ctx->pinned, 0) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(ctx->pinned);
        delete ctx;
        return SCCG_ECUDA;
    }
    if (cudaMalloc(&ctx->counters, sizeof(WorkCounters)) != cudaSuccess ||
        cudaMemset(ctx->counters, 0, sizeof(WorkCounters)) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(ctx->pinned);
        delete ctx;
        return SCCG_ENOMEM;
    }
    if (cudaStreamCreateWithFlags(&ctx->side_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->fork_event, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&ctx->join_event, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        sccg_ctx_destroy(ctx);
        return SCCG_ECUDA;
    }
    *out = ctx;
    return SCCG_OK;
}

int sccg_ctx_destroy(sccg_ctx* ctx)
{
    if (!ctx) return SCCG_EINVAL;
    {
        DeviceGuard g(ctx->device);
        cudaDeviceSynchronize();
        if (ctx->ws) cudaFree(ctx->ws);
        for (int k = 0; k < 4; ++k)
            if (ctx->aux[k]) cudaFree(ctx->aux[k]);
        if (ctx->counters) cudaFree(ctx->counters);
        if (ctx->pinned) cudaFreeHost(ctx->pinned);
        if (ctx->batch_exec) cudaGraphExecDestroy(ctx->batch_exec);
        if (ctx->side_stream) cudaStreamDestroy(ctx->side_stream);
        if (ctx->fork_event) cudaEventDestroy(ctx->fork_event);
        if (ctx->join_event) cudaEventDestroy(ctx->join_event);
        if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
        if (ctx->tile_streams_ready) {
            for (int k = 0; k < sccg_ctx::kTileStreams; ++k) cudaStreamDestroy(ctx->tstream[k]);
            for (int k = 0; k <= sccg_ctx::kTileStreams; ++k) cudaEventDestroy(ctx->tevent[k]);
        }
    }
    delete ctx;
    return SCCG_OK;
}

int sccg_ctx_set_param(sccg_ctx* ctx, const char* name, int64_t value)
{
    if (!ctx || !name) return SCCG_EINVAL;
    sccg_params p = ctx->params;
    if (!strcmp(name, "T")) p.T = (int32_t)value;
    else if (!strcmp(name, "warps_per_cta")) p.warps_per_cta = (int32_t)value;
    else if (!strcmp(name, "split_pixels")) p.split_pixels = (int32_t)value;
    else if (!strcmp(name, "ctas_per_sm")) p.ctas_per_sm = (int32_t)value;
    else if (!strcmp(name, "area_method")) p.area_method = (int32_t)value;
    else if (!strcmp(name, "leaf_words")) p.leaf_words = (int32_t)value;
    else if (!strcmp(name, "pair_lanes")) p.pair_lanes = (int32_t)value;
    else if (!strcmp(name, "area_T")) p.area_T = (int32_t)value;
    else if (!strcmp(name, "rasters")) p.rasters = (int32_t)value;
    else if (!strcmp(name, "raster_heavy")) p.raster_heavy = (int32_t)value;
    else if (!strcmp(name, "raster_lanes")) p.raster_lanes = (int32_t)value;
    else if (!strcmp(name, "count_work")) { ctx->count_work = value != 0; return SCCG_OK; }
    else if (!strcmp(name, "candidate_speculative")) {
        if (value < 0 || value > 2) return SCCG_EINVAL;
        ctx->cand_speculative = (int)value;
        return SCCG_OK;
    }
    else return SCCG_EINVAL;
    const int r = validate_params(p);
    if (r) return r;
    ctx->params = p;
    return SCCG_OK;
}

int sccg_ctx_reserve(sccg_ctx* ctx, int64_t max_pairs)
{
    if (!ctx || max_pairs < 0) return SCCG_EINVAL;
    if (max_pairs >= kJaccardMaxPairs) return SCCG_ERANGE;
    DeviceGuard g(ctx->device);
    return ws_reserve(ctx, std::max(persistent_scratch(std::max<long long>(max_pairs, 1)),
                                    jaccard_scratch(ctx, max_pairs)));
}

int sccg_ctx_get_params(const sccg_ctx* ctx, sccg_params* out)
{
    if (!ctx || !out) return SCCG_EINVAL;
    *out = ctx->params;
    return SCCG_OK;
}

const char* sccg_last_error(const sccg_ctx* ctx) { return ctx ? ctx->last_err : ""; }

int sccg_work_counters(sccg_ctx* ctx, uint64_t* out12, int reset)
{
    if (!ctx || !out12) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    WorkCounters h;
    SCCG_CUDA(ctx, cudaMemcpy(&h, ctx->counters, sizeof h, cudaMemcpyDeviceToHost));
    out12[0] = h.strip_edges; out12[1] = h.pixel_edges; out12[2] = h.box_edges; out12[3] = h.boxes;
    out12[4] = h.row_entries; out12[5] = h.row_edges; out12[6] = h.scan_entries; out12[7] = h.scan_pairs;
    out12[8] = h.leaf_pixels; out12[9] = h.window_pixels; out12[10] = h.raster_out; out12[11] = h.raster_and;
    if (reset) SCCG_CUDA(ctx, cudaMemset(ctx->counters, 0, sizeof(WorkCounters)));
    return SCCG_OK;
}

int sccg_prepare_sets(sccg_ctx* ctx, sccg_polyset* sets, int n_sets, void* stream)
{
    if (!ctx || !sets || n_sets < 1 || n_sets > kMaxPrepSets) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    size_t need = carve_size<PrepStats>(n_sets);
    long long max_n = 0;
    for (int k = 0; k < n_sets; ++k) {
        sccg_polyset* s = sets + k;
        if (s->n < 0 || s->n > 0x7fffffffLL) return SCCG_EINVAL;
        s->reserved = 0;
        if (!is_device_ptr(s->off) || !is_device_ptr(s->mbr) || !is_device_ptr(s->area)) return SCCG_EINVAL;
        if (s->n > 0 && !is_device_ptr(s->xy)) return SCCG_EINVAL;
        if (s->tile && !is_device_ptr(s->tile)) return SCCG_EINVAL;
        if (reinterpret_cast<uintptr_t>(s->xy) % 8 || reinterpret_cast<uintptr_t>(s->mbr) % 16) return SCCG_EINVAL;
        s->raster_ok = 0;
        s->raster_bytes = 0;
        if (s->raster && (!is_device_ptr(s->raster) || reinterpret_cast<uintptr_t>(s->raster) % 16 || s->raster_cap < 0))
            return SCCG_EINVAL;
        need += carve_size<int>(s->n + 1);
        if (s->raster) need += carve_size<long long>(s->n + 1) + carve_size<long long>(s->n / kScanBlock + 2);
        max_n = std::max<long long>(max_n, s->n);
    }
    need += band_build_scratch(max_n);     // for the band index of deferred polygons, after the sync
    int r = ws_reserve(ctx, need);
    if (r) return r;
    Carve cv(ctx->ws);
    PrepStats* stats = cv.take<PrepStats>(n_sets);
    int* big_lists[kMaxPrepSets];
    const PrepStats init{0, 0, 0, 0, 0x7fffffffffffffffLL, 0, 0};
    // the initial stats are copied from pinned memory by a kernel, kept ordered on the stream
    static_assert(sizeof(PrepStats) % 8 == 0, "prepare stats are copied in 8-byte words");
    PrepStats* hstats = static_cast<PrepStats*>(ctx->pinned);
    for (int k = 0; k < n_sets; ++k) hstats[k] = init;
    r = small_copy(ctx, stats, ctx->pinned_dev, n_sets * sizeof init, st);
    if (r) return r;
    // odd-numbered sets run on the side stream, beside the even ones (one fork, one join)
    const bool two_streams = n_sets > 1;
    if (two_streams) {
        SCCG_CUDA(ctx, cudaEventRecord(ctx->fork_event, st));
        SCCG_CUDA(ctx, cudaStreamWaitEvent(ctx->side_stream, ctx->fork_event, 0));
    }
    long long* roffs[kMaxPrepSets];
    long long* rscan[kMaxPrepSets];
    long long* rbsum[kMaxPrepSets];
    bool rleaf[kMaxPrepSets];
    for (int k = 0; k < n_sets; ++k) {
        const sccg_polyset* s = sets + k;
        int* big_list = big_lists[k] = cv.take<int>(s->n + 1);
        unsigned* big_n = &stats[k].deferred;
        cudaStream_t sk = (two_streams && (k & 1)) ? ctx->side_stream : st;
        roffs[k] = nullptr;
        if (s->raster && s->n > 0) {
            // one pass: MBR, validation, and the leaf windows pixelized into their raster slots; the
            // larger windows are listed and drawn after the synchronisation
            const long long hb = raster_head_bytes(s->n);
            rscan[k] = cv.take<long long>(s->n + 1);
            rbsum[k] = cv.take<long long>(s->n / kScanBlock + 2);
            rleaf[k] = s->raster_cap >= hb + 4LL * kRasterSlot * s->n;
            roffs[k] = static_cast<long long*>(s->raster);
            PrepArgs a{s->n, s->off, s->xy, s->tile, reinterpret_cast<int4*>(s->mbr), s->area, stats + k,
                       ctx->params.area_T, ctx->counters, 0, big_list, big_n, ctx->params.leaf_words, 0,
                       rleaf[k] ? roffs[k] : nullptr,
                       rleaf[k] ? reinterpret_cast<uint32_t*>(static_cast<char*>(s->raster) + hb) : nullptr,
                       rleaf[k] ? 1 : 0};
            r = launch_prepare<kCapSmall, true, true>(ctx, a, sk);
            if (r) return r;
        } else if (s->n > 0 && ctx->params.area_method != SCCG_AREA_PIXELBOX) {
            // polygons counted by rows are listed and counted after the sync (k_area_bands)
            PrepArgs a{s->n, s->off, s->xy, s->tile, reinterpret_cast<int4*>(s->mbr), s->area, stats + k,
                       ctx->params.area_T, ctx->counters, 0, big_list, big_n, ctx->params.leaf_words,
                       ctx->params.area_method == SCCG_AREA_SHOELACE ? 1 : 0};
            r = launch_prepare<kCapSmall, true>(ctx, a, sk);
            if (r) return r;
        } else if (s->n > 0) {
            PrepArgs a{s->n, s->off, s->xy, s->tile, reinterpret_cast<int4*>(s->mbr), s->area, stats + k,
                       ctx->params.T, ctx->counters, kCapSmall, big_list, big_n, ctx->params.leaf_words};
            // polygons with more than kCapSmall vertices are listed and done with the larger buffers
            r = launch_prepare<kCapSmall, false>(ctx, a, sk);
            if (r) return r;
            r = launch_prepare_big<kCapBig>(ctx, a, sk);
            if (r) return r;
        }
    }
    if (two_streams) {
        SCCG_CUDA(ctx, cudaEventRecord(ctx->join_event, ctx->side_stream));
        SCCG_CUDA(ctx, cudaStreamWaitEvent(st, ctx->join_event, 0));
    }
    const Carve after_lists = cv;        // scratch of the band builds below starts here
    r = small_copy(ctx, ctx->pinned_dev, stats, n_sets * sizeof init, st);
    if (r) return r;
    SCCG_CUDA(ctx, cudaStreamSynchronize(st));
    int status = SCCG_OK;
    for (int k = 0; k < n_sets; ++k) {
        sccg_polyset* s = sets + k;
        const PrepStats res = hstats[k];
        s->max_nv = res.max_nv;
        s->max_extent = res.max_extent;
        s->n_tiles = std::max(res.n_tiles, s->n > 0 ? 1 : 0);
        s->band_bytes = res.band_bytes ? band_head_bytes(s->n) + (long long)res.band_bytes : 0;
        s->bands = nullptr;
        const bool rasters = roffs[k] != nullptr;
        if (rasters) {
            s->raster_bytes = raster_head_bytes(s->n) + 4 * (kRasterSlot * s->n + (long long)res.raster_words);
            s->raster_ok = !res.err && rleaf[k] && s->raster_bytes <= s->raster_cap ? 1 : 0;
            if (s->raster_ok) {
                // the listed (larger) rasters after the slots, in list order
                const unsigned nl = res.deferred;
                const unsigned g = (unsigned)std::max<long long>(1, std::min<long long>((nl + 255) / 256, 4LL * ctx->sm_count));
                k_raster_sizes<<<g, 256, 0, st>>>(big_lists[k], &stats[k].deferred, reinterpret_cast<const int4*>(s->mbr),
                                                  rscan[k]);
                int rr = device_scan(ctx, rscan[k], nl, rscan[k], rbsum[k], st);
                if (rr) return rr;
                k_raster_place<<<g, 256, 0, st>>>(big_lists[k], &stats[k].deferred, rscan[k], s->n, roffs[k]);
                SCCG_LAUNCHED(ctx, "k_raster_place");
                ctx->launches += 2;
            }
        }
        if (!res.err && res.deferred && (rasters || ctx->params.area_method != SCCG_AREA_PIXELBOX)) {
            // areas of the deferred polygons by rows; those with 1024 or more vertices from a
            // temporary band index
            int rr = SCCG_OK;
            const char* blob = nullptr;
            if (s->band_bytes) {
                rr = aux_reserve(ctx, 2, (size_t)s->band_bytes);
                Carve bcv = after_lists;
                if (!rr) rr = build_bands_into(ctx, s, static_cast<char*>(ctx->aux[2]), s->band_bytes, bcv, st);
                blob = static_cast<const char*>(ctx->aux[2]);
            }
            if (!rr && s->raster_ok) {
                // rasters of the windows over 64 pixels wide or high, and their areas: those drawn from
                // their rings, then (when the set has a band index) those drawn band by band
                uint32_t* rw = reinterpret_cast<uint32_t*>(static_cast<char*>(s->raster) + raster_head_bytes(s->n));
                const int4* mbr = reinterpret_cast<const int4*>(s->mbr);
                // (the ring instance's warps take the listed polygons from a counter, stats[k].next, zero
                // since the stats were initialised at the start of this call)
                rr = launch_raster_big<32, false>(ctx, s, blob, big_lists[k], &stats[k].deferred, res.deferred,
                                                  roffs[k], rw, mbr, &stats[k].next, st);
                if (!rr && blob)
                    rr = launch_raster_big<64, true>(ctx, s, blob, big_lists[k], &stats[k].deferred, res.deferred,
                                                     roffs[k], rw, mbr, nullptr, st);
            } else if (!rr) {
                const int wpc = 4;
                const size_t smem = sizeof(ScanSmem) * wpc;
                auto kfn = ctx->count_work ? k_area_bands<true> : k_area_bands<false>;
                const unsigned grid = (unsigned)((res.deferred + wpc - 1) / wpc);
                kfn<<<grid, 32 * wpc, smem, st>>>(s->off, s->xy, reinterpret_cast<const int4*>(s->mbr), blob,
                                                  big_lists[k], &stats[k].deferred, s->area, ctx->counters);
                SCCG_LAUNCHED(ctx, "k_area_bands");
                ctx->launches += 1;
            }
            if (rr && !status) status = rr;
        }
        if (res.err & (kErrFewVertices | kErrTiles)) {
            snprintf(ctx->last_err, sizeof ctx->last_err,
                     "invalid polygon set %d (flags %d, first bad polygon %lld)", k, res.err, res.first_bad);
            if (!status) status = SCCG_EINVAL;
        } else if (res.err & kErrRange) {
            snprintf(ctx->last_err, sizeof ctx->last_err, "set %d: coordinate/extent out of range at polygon %lld",
                     k, res.first_bad);
            if (!status) status = SCCG_ERANGE;
        } else {
            s->reserved = (int32_t)kPreparedMagic;
        }
    }
    return status;
}

int sccg_raster_bytes(sccg_ctx* ctx, sccg_polyset* s, int64_t* bytes, void* stream)
{
    if (!ctx || !s || !bytes) return SCCG_EINVAL;
    if (s->n < 0 || s->n > 0x7fffffffLL) return SCCG_EINVAL;
    if (!is_device_ptr(s->off) || !is_device_ptr(s->mbr)) return SCCG_EINVAL;
    if (s->n > 0 && !is_device_ptr(s->xy)) return SCCG_EINVAL;
    if (s->tile && !is_device_ptr(s->tile)) return SCCG_EINVAL;
    if (reinterpret_cast<uintptr_t>(s->xy) % 8 || reinterpret_cast<uintptr_t>(s->mbr) % 16) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const long long n = s->n;
    int r = ws_reserve(ctx, carve_size<PrepStats>(1) + carve_size<long long>(n + 1) +
                                carve_size<long long>(n / kScanBlock + 2));
    if (r) return r;
    Carve cv(ctx->ws);
    PrepStats* stats = cv.take<PrepStats>(1);
    long long* words = cv.take<long long>(n + 1);
    long long* bsum = cv.take<long long>(n / kScanBlock + 2);
    PrepStats* hstats = static_cast<PrepStats*>(ctx->pinned);
    *hstats = PrepStats{0, 0, 0, 0, 0x7fffffffffffffffLL, 0, 0};
    r = small_copy(ctx, stats, ctx->pinned_dev, sizeof(PrepStats), st);
    if (r) return r;
    PrepArgs a{n, s->off, s->xy, s->tile, reinterpret_cast<int4*>(s->mbr), s->area, stats};
    if (n > 0) {
        r = launch_mbr(ctx, a, words, st);
        if (!r) r = device_scan(ctx, words, n, words, bsum, st);
    } else {
        r = zero_async(ctx, words, sizeof(long long), st);
    }
    if (!r) r = small_copy(ctx, ctx->pinned_dev, stats, sizeof(PrepStats), st);
    if (!r) r = small_copy(ctx, static_cast<char*>(ctx->pinned_dev) + sizeof(PrepStats), words + n, 8, st);
    if (r) return r;
    SCCG_CUDA(ctx, cudaStreamSynchronize(st));
    const PrepStats res = *hstats;
    const long long total = *reinterpret_cast<const long long*>(static_cast<const char*>(ctx->pinned) + sizeof(PrepStats));
    if (res.err & (kErrFewVertices | kErrTiles)) {
        snprintf(ctx->last_err, sizeof ctx->last_err, "invalid polygon set (flags %d, first bad polygon %lld)",
                 res.err, res.first_bad);
        return SCCG_EINVAL;
    }
    if (res.err & kErrRange) {
        snprintf(ctx->last_err, sizeof ctx->last_err, "coordinate/extent out of range at polygon %lld", res.first_bad);
        return SCCG_ERANGE;
    }
    *bytes = raster_head_bytes(n) + 4 * (kRasterSlot * n + total);
    return SCCG_OK;
}

int sccg_prepare(sccg_ctx* ctx, sccg_polyset* s, void* stream)
{
    if (!ctx || !s) return SCCG_EINVAL;
    return sccg_prepare_sets(ctx, s, 1, stream);
}

int sccg_build_bands(sccg_ctx* ctx, sccg_polyset* s, void* buf, int64_t bytes, void* stream)
{
    if (!ctx || check_prepared(s)) return SCCG_EINVAL;
    if (s->band_bytes == 0) {
        s->bands = nullptr;
        return SCCG_OK;
    }
    if (bytes < s->band_bytes) return SCCG_ECAPACITY;
    if (!buf || !is_device_ptr(buf) || reinterpret_cast<uintptr_t>(buf) % 16) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int r = ws_reserve(ctx, band_build_scratch(s->n));
    if (r) return r;
    Carve cv(ctx->ws);
    r = build_bands_into(ctx, s, static_cast<char*>(buf), s->band_bytes, cv, st);
    if (r) return r;
    s->bands = buf;
    return SCCG_OK;
}

// Candidate pairs (validated arguments). spec: size the grid buffers from cells_per_b and
// entries_per_b instead of synchronising on their counts; *fits = false then means they were too
// small and nothing was written. *ncell_out / *nent_out: the sizes used (the exact counts when !spec).
int candidate_pairs_run(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, int32_t* pa, int32_t* pb,
                        int64_t capacity, int64_t* n_pairs, int64_t* tile_pair_off, bool tpo_host, cudaStream_t st,
                        bool spec, double cells_per_b, double entries_per_b, bool* fits, long long* ncell_out,
                        long long* nent_out)
{
    const int n_tiles = std::max(std::max(A->n_tiles, B->n_tiles), 1);
    const long long nA = A->n, nB = B->n;
    const long long nscan = std::max<long long>(std::max(nA, (long long)n_tiles), 1);
    const long long nb = (nscan + kScanBlock - 1) / kScanBlock + 1;
    const size_t need = carve_size<long long>(n_tiles + 1) * 5 + carve_size<TileGrid>(n_tiles) +
                        carve_size<long long>(nA + 1) * 2 + carve_size<long long>(nb) +
                        carve_size<int>(nA + 1) * 2 + carve_size<unsigned long long>(4) +
                        carve_size<unsigned long long>(1);
    int r = ws_reserve(ctx, need);
    if (r) return r;
    Carve cv(ctx->ws);
    long long* astart = cv.take<long long>(n_tiles + 1);
    long long* bstart = cv.take<long long>(n_tiles + 1);
    long long* ncells = cv.take<long long>(n_tiles + 1);
    long long* cellbase = cv.take<long long>(n_tiles + 1);
    TileGrid* grid = cv.take<TileGrid>(n_tiles);
    long long* tpo_dev = cv.take<long long>(n_tiles + 1);
    long long* counts = cv.take<long long>(nA + 1);
    long long* offs = cv.take<long long>(nA + 1);
    long long* bsum = cv.take<long long>(nb);
    int* big_list = cv.take<int>(nA + 1);
    int* mid_list = cv.take<int>(nA + 1);
    unsigned long long* small = cv.take<unsigned long long>(4);   // [0] big count, [1] mid count (as unsigned)
    unsigned long long* ok = spec ? cv.take<unsigned long long>(1) : nullptr;
    long long* h = static_cast<long long*>(ctx->pinned);
    const int4* mA = reinterpret_cast<const int4*>(A->mbr);
    const int4* mB = reinterpret_cast<const int4*>(B->mbr);
    const unsigned tg = (unsigned)((n_tiles + 1 + 255) / 256);
    k_tile_ranges<<<tg, 256, 0, st>>>(A->tile, nA, n_tiles, astart);
    k_tile_ranges<<<tg, 256, 0, st>>>(B->tile, nB, n_tiles, bstart);
    k_tile_grid<<<(unsigned)((32LL * n_tiles + 255) / 256), 256, 0, st>>>(mB, bstart, n_tiles, grid, ncells);
    SCCG_LAUNCHED(ctx, "k_tile_grid");
    ctx->launches += 3;
    r = device_scan(ctx, ncells, n_tiles, cellbase, bsum, st);
    if (r) return r;
    long long ncell = 0;
    if (spec) {
        ncell = cells_per_b < 0 ? 1 : (long long)(cells_per_b * (double)nB) + 64LL * n_tiles + 1024;
        k_cap_check<<<1, 32, 0, st>>>(cellbase + n_tiles, ncell, ok, 1);
        SCCG_LAUNCHED(ctx, "k_cap_check");
        ctx->launches += 1;
    } else {
        // 1st sync: number of grid cells
        r = small_copy(ctx, ctx->pinned_dev, cellbase + n_tiles, sizeof(long long), st);
        if (r) return r;
        SCCG_CUDA(ctx, cudaStreamSynchronize(st));
        ncell = *h;
    }
    const long long nbc = (std::max(ncell, 1LL) + kScanBlock - 1) / kScanBlock + 1;
    r = aux_reserve(ctx, 0, carve_size<unsigned long long>(ncell + 1) + carve_size<long long>(ncell + 1) +
                                carve_size<int>(ncell + 1) + carve_size<long long>(nbc));
    if (r) return r;
    Carve ca(ctx->aux[0]);
    unsigned long long* ccount = ca.take<unsigned long long>(ncell + 1);
    long long* cell_off = ca.take<long long>(ncell + 1);
    int* cursor = ca.take<int>(ncell + 1);
    long long* bsum2 = ca.take<long long>(nbc);
    r = zero_async(ctx, ccount, sizeof(unsigned long long) * (ncell + 1), st);
    if (!r) r = zero_async(ctx, cursor, sizeof(int) * (ncell + 1), st);
    if (r) return r;
    const unsigned gb = (unsigned)((std::max(nB, 1LL) + 255) / 256);
    if (nB > 0) {
        k_bin_count<<<gb, 256, 0, st>>>(mB, B->tile, nB, grid, cellbase, ccount, ok);
        SCCG_LAUNCHED(ctx, "k_bin_count");
        ctx->launches += 1;
    }
    r = device_scan(ctx, reinterpret_cast<const long long*>(ccount), ncell, cell_off, bsum2, st);
    if (r) return r;
    long long nent = 0;
    if (spec) {
        nent = entries_per_b < 0 ? 1 : (long long)(entries_per_b * (double)nB) + 1024;
        k_cap_check<<<1, 32, 0, st>>>(cell_off + ncell, nent, ok, 0);
        SCCG_LAUNCHED(ctx, "k_cap_check");
        ctx->launches += 1;
    } else {
        // 2nd sync: number of cell registrations
        r = small_copy(ctx, ctx->pinned_dev, cell_off + ncell, sizeof(long long), st);
        if (r) return r;
        SCCG_CUDA(ctx, cudaStreamSynchronize(st));
        nent = *h;
    }
    *ncell_out = ncell;
    *nent_out = nent;
    r = aux_reserve(ctx, 1, carve_size<int>(nent + 1));
    if (r) return r;
    int* entries = static_cast<int*>(ctx->aux[1]);
    if (nB > 0) {
        k_bin_fill<<<gb, 256, 0, st>>>(mB, B->tile, nB, grid, cellbase, cursor, cell_off, entries, ok);
        SCCG_LAUNCHED(ctx, "k_bin_fill");
        ctx->launches += 1;
    }
    ProbeArgs pr{mA, A->tile, nA, mB, grid, cellbase, cell_off, entries, n_tiles, ok};
    r = zero_async(ctx, small, sizeof(unsigned long long) * 4, st);
    if (r) return r;
    unsigned* big_n = reinterpret_cast<unsigned*>(small);
    unsigned* mid_n = reinterpret_cast<unsigned*>(small + 1);
    const unsigned ga = (unsigned)((std::max(nA, 1LL) + 255) / 256);
    r = aux_reserve(ctx, 3, sizeof(int) * (size_t)kSmallPairs * (size_t)std::max(nA, 1LL));
    if (r) return r;
    int* cand = static_cast<int*>(ctx->aux[3]);
    if (nA > 0) {
        k_probe_count<<<ga, 256, 0, st>>>(pr, counts, big_list, big_n, cand, mid_list, mid_n);
        k_probe_count_mid<<<(unsigned)(8 * ctx->sm_count), 256, 0, st>>>(pr, mid_list, mid_n, counts, big_list, big_n,
                                                                        cand);
        k_probe_count_big<<<(unsigned)(2 * ctx->sm_count), 256, 0, st>>>(pr, big_list, big_n, counts);
        SCCG_LAUNCHED(ctx, "k_probe_count");
        ctx->launches += 3;
    }
    r = device_scan(ctx, counts, nA, offs, bsum, st);
    if (r) return r;
    if (nA > 0 && capacity > 0) {
        k_probe_emit_small<<<ga, 256, 0, st>>>(nA, offs, cand, pa, pb, capacity);
        k_probe_write_big<<<(unsigned)(2 * ctx->sm_count), 256, 0, st>>>(pr, bstart, offs, big_list, big_n, pa, pb,
                                                                        capacity);
        SCCG_LAUNCHED(ctx, "k_probe_write");
        ctx->launches += 2;
    }
    if (tile_pair_off) {
        k_gather_tile_offsets<<<tg, 256, 0, st>>>(offs, astart, n_tiles, n_tiles, nA,
                                                  tpo_host ? reinterpret_cast<int64_t*>(tpo_dev) : tile_pair_off);
        SCCG_LAUNCHED(ctx, "k_gather_tile_offsets");
        ctx->launches += 1;
    }
    r = small_copy(ctx, ctx->pinned_dev, offs + nA, sizeof(long long), st);
    if (!r && spec) r = small_copy(ctx, static_cast<char*>(ctx->pinned_dev) + 8, ok, sizeof(unsigned long long), st);
    if (r) return r;
    if (tpo_host)
        SCCG_CUDA(ctx, cudaMemcpyAsync(tile_pair_off, tpo_dev, sizeof(long long) * (n_tiles + 1),
                                       cudaMemcpyDeviceToHost, st));
    // last (with spec, only) sync: number of pairs
    SCCG_CUDA(ctx, cudaStreamSynchronize(st));
    *n_pairs = h[0];
    *fits = !spec || h[1] != 0;
    if (!*fits) return SCCG_OK;
    return h[0] > capacity ? SCCG_ECAPACITY : SCCG_OK;
}

int sccg_candidate_pairs(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, int32_t* pa,
                         int32_t* pb, int64_t capacity, int64_t* n_pairs, int64_t* tile_pair_off,
                         void* stream)
{
    if (!ctx || !n_pairs || capacity < 0) return SCCG_EINVAL;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (capacity > 0 && (!is_device_ptr(pa) || !is_device_ptr(pb))) return SCCG_EINVAL;
    const bool tpo_host = tile_pair_off && !is_device_ptr(tile_pair_off);
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int mode = ctx->cand_speculative;
    bool fits = true;
    long long ncell = 0, nent = 0;
    if (mode) {
        const double cpb = mode == 2 ? -1.0 : ctx->cand_cells_per_b;
        const double epb = mode == 2 ? -1.0 : ctx->cand_entries_per_b;
        const int r = candidate_pairs_run(ctx, A, B, pa, pb, capacity, n_pairs, tile_pair_off, tpo_host, st, true, cpb,
                                          epb, &fits, &ncell, &nent);
        if (r || fits) return r;
    }
    // the buffers were too small (or sizing by counts was asked for): exact sizes, then remember them
    const int r = candidate_pairs_run(ctx, A, B, pa, pb, capacity, n_pairs, tile_pair_off, tpo_host, st, false, 0.0,
                                      0.0, &fits, &ncell, &nent);
    if ((r == SCCG_OK || r == SCCG_ECAPACITY) && mode == 1 && B->n > 0) {
        ctx->cand_cells_per_b = std::max(ctx->cand_cells_per_b, 1.25 * (double)ncell / (double)B->n);
        ctx->cand_entries_per_b = std::max(ctx->cand_entries_per_b, 1.25 * (double)nent / (double)B->n);
    }
    return r;
}

int sccg_pair_areas(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa,
                    const int32_t* pb, int64_t n_pairs, int64_t* inter, int64_t* uni, int mode, void* stream)
{
    if (!ctx || n_pairs < 0) return SCCG_EINVAL;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (mode != SCCG_MODE_PLAIN && mode != SCCG_MODE_PERSISTENT && mode != SCCG_MODE_NOSEP) return SCCG_EINVAL;
    if (mode == SCCG_MODE_NOSEP && std::max(A->max_extent, B->max_extent) > kNoSepExtent) return SCCG_ERANGE;
    if (n_pairs == 0) return SCCG_OK;
    if (!is_device_ptr(pa) || !is_device_ptr(pb) || !is_device_ptr(inter) || !is_device_ptr(uni))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AreasArgs a{n_pairs, A->n, B->n, pa, pb,
                A->off, A->xy, reinterpret_cast<const int4*>(A->mbr), A->area,
                B->off, B->xy, reinterpret_cast<const int4*>(B->mbr), B->area,
                inter, uni, ctx->params.T, ctx->counters,
                static_cast<const char*>(A->bands), static_cast<const char*>(B->bands),
                ctx->params.leaf_words};
    if (mode != SCCG_MODE_NOSEP) use_rasters(ctx, A, B, a);
    const int cap = edge_cap_for(std::max(A->max_nv, B->max_nv));
    if (mode == SCCG_MODE_PERSISTENT) {
        const int r = ws_reserve(ctx, persistent_scratch(n_pairs));
        if (r) return r;
        return persistent_launch(ctx, a, cap, st);
    }
    if (mode == SCCG_MODE_NOSEP)
        return cap == kCapSmall ? launch_plain<kCapSmall, true>(ctx, a, st) : launch_plain<kCapBig, true>(ctx, a, st);
    return cap == kCapSmall ? launch_plain<kCapSmall>(ctx, a, st) : launch_plain<kCapBig>(ctx, a, st);
}

int sccg_pair_areas_tiles(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa,
                          const int32_t* pb, const int64_t* tile_pair_off, int32_t n_tiles, int64_t* inter,
                          int64_t* uni, void* stream)
{
    if (!ctx || !tile_pair_off || n_tiles < 0) return SCCG_EINVAL;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (is_device_ptr(tile_pair_off)) return SCCG_EINVAL;   // must be host memory
    if (n_tiles == 0 || tile_pair_off[n_tiles] == 0) return SCCG_OK;
    if (tile_pair_off[0] != 0) return SCCG_EINVAL;
    for (int t = 0; t < n_tiles; ++t)
        if (tile_pair_off[t + 1] < tile_pair_off[t]) return SCCG_EINVAL;
    if (!is_device_ptr(pa) || !is_device_ptr(pb) || !is_device_ptr(inter) || !is_device_ptr(uni))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (!ctx->tile_streams_ready) {
        for (int k = 0; k < sccg_ctx::kTileStreams; ++k)
            SCCG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->tstream[k], cudaStreamNonBlocking));
        for (int k = 0; k <= sccg_ctx::kTileStreams; ++k)
            SCCG_CUDA(ctx, cudaEventCreateWithFlags(&ctx->tevent[k], cudaEventDisableTiming));
        ctx->tile_streams_ready = true;
    }
    // fork the tile streams from the caller's stream
    SCCG_CUDA(ctx, cudaEventRecord(ctx->tevent[sccg_ctx::kTileStreams], st));
    for (int k = 0; k < sccg_ctx::kTileStreams; ++k)
        SCCG_CUDA(ctx, cudaStreamWaitEvent(ctx->tstream[k], ctx->tevent[sccg_ctx::kTileStreams], 0));
    const int cap = edge_cap_for(std::max(A->max_nv, B->max_nv));
    int k = 0;
    for (int t = 0; t < n_tiles; ++t) {
        const long long p0 = tile_pair_off[t], p1 = tile_pair_off[t + 1];
        if (p1 == p0) continue;
        AreasArgs a{p1 - p0, A->n, B->n, pa + p0, pb + p0,
                    A->off, A->xy, reinterpret_cast<const int4*>(A->mbr), A->area,
                    B->off, B->xy, reinterpret_cast<const int4*>(B->mbr), B->area,
                    inter + p0, uni + p0, ctx->params.T, ctx->counters,
                    static_cast<const char*>(A->bands), static_cast<const char*>(B->bands),
                    ctx->params.leaf_words};
        use_rasters(ctx, A, B, a);
        int r;
        r = cap == kCapSmall ? launch_plain<kCapSmall>(ctx, a, ctx->tstream[k])
                             : launch_plain<kCapBig>(ctx, a, ctx->tstream[k]);
        if (r) return r;
        k = (k + 1) % sccg_ctx::kTileStreams;
    }
    // join them back into the caller's stream
    for (int j = 0; j < sccg_ctx::kTileStreams; ++j) {
        SCCG_CUDA(ctx, cudaEventRecord(ctx->tevent[j], ctx->tstream[j]));
        SCCG_CUDA(ctx, cudaStreamWaitEvent(st, ctx->tevent[j], 0));
    }
    return SCCG_OK;
}

int sccg_batch_run(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa,
                   const int32_t* pb, int64_t n_pairs, int64_t* inter, int64_t* uni, sccg_jaccard_result* out,
                   void* stream)
{
    if (!ctx || !out || n_pairs < 0) return SCCG_EINVAL;
    if (n_pairs >= kJaccardMaxPairs) return SCCG_ERANGE;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (!is_device_ptr(out)) return SCCG_EINVAL;
    if (n_pairs > 0 && (!is_device_ptr(pa) || !is_device_ptr(pb) || !is_device_ptr(inter) || !is_device_ptr(uni)))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int r = ws_reserve(ctx, std::max(persistent_scratch(std::max<long long>(n_pairs, 1)), jaccard_scratch(ctx, n_pairs)));
    if (r) return r;
    const void* key[13] = {A->off, A->xy, A->mbr, A->bands, B->off, B->xy, B->mbr, B->bands, pa, inter, out,
                           A->raster_ok ? A->raster : nullptr, B->raster_ok ? B->raster : nullptr};
    const bool same = ctx->batch_exec && ctx->batch_n == n_pairs && !memcmp(key, ctx->batch_key, sizeof key) &&
                      !memcmp(&ctx->batch_params, &ctx->params, sizeof(sccg_params)) &&
                      ctx->batch_count_work == ctx->count_work && ctx->batch_key[0] != nullptr;
    if (!same) {
        if (ctx->batch_exec) {
            cudaGraphExecDestroy(ctx->batch_exec);
            ctx->batch_exec = nullptr;
        }
        if (!ctx->cap_stream) SCCG_CUDA(ctx, cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        AreasArgs a{n_pairs, A->n, B->n, pa, pb,
                    A->off, A->xy, reinterpret_cast<const int4*>(A->mbr), A->area,
                    B->off, B->xy, reinterpret_cast<const int4*>(B->mbr), B->area,
                    inter, uni, ctx->params.T, ctx->counters,
                static_cast<const char*>(A->bands), static_cast<const char*>(B->bands),
                ctx->params.leaf_words};
        use_rasters(ctx, A, B, a);
        const int cap = edge_cap_for(std::max(A->max_nv, B->max_nv));
        const unsigned long long launches0 = ctx->launches;
        SCCG_CUDA(ctx, cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        r = n_pairs > 0 ? persistent_launch(ctx, a, cap, ctx->cap_stream) : SCCG_OK;
        if (!r) r = jaccard_launch(ctx, inter, uni, n_pairs, reinterpret_cast<JaccardOut*>(out), ctx->cap_stream);
        cudaGraph_t graph = nullptr;
        const cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &graph);
        ctx->batch_launches = ctx->launches - launches0;     // kernels in the graph
        ctx->launches = launches0;
        if (r) {
            if (graph) cudaGraphDestroy(graph);
            return r;
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
        const cudaError_t ei = cudaGraphInstantiate(&ctx->batch_exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ei != cudaSuccess) {
            ctx->batch_exec = nullptr;
            return cuda_fail(ctx, ei, "cudaGraphInstantiate");
        }
        memcpy(ctx->batch_key, key, sizeof key);
        ctx->batch_n = n_pairs;
        ctx->batch_params = ctx->params;
        ctx->batch_count_work = ctx->count_work;
    }
    SCCG_CUDA(ctx, cudaGraphLaunch(ctx->batch_exec, st));
    ctx->launches += ctx->batch_launches;
    return SCCG_OK;
}

int sccg_rebase_pairs(sccg_ctx* ctx, int32_t* pa, int32_t* pb, int64_t n_pairs, int64_t base_a, int64_t base_b,
                      void* stream)
{
    if (!ctx || n_pairs < 0 || base_a < 0 || base_b < 0 || base_a > 0x7fffffffLL || base_b > 0x7fffffffLL)
        return SCCG_EINVAL;
    if (n_pairs == 0) return SCCG_OK;
    if (!is_device_ptr(pa) || !is_device_ptr(pb)) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)std::min<long long>((n_pairs + 255) / 256, 8LL * ctx->sm_count);
    k_rebase_pairs<<<grid, 256, 0, st>>>(pa, pb, n_pairs, (int)base_a, (int)base_b);
    SCCG_LAUNCHED(ctx, "k_rebase_pairs");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_contains(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa, const int32_t* pb,
                  const int64_t* inter, int64_t n_pairs, uint8_t* out, void* stream)
{
    if (!ctx || n_pairs < 0) return SCCG_EINVAL;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (n_pairs == 0) return SCCG_OK;
    if (!is_device_ptr(pa) || !is_device_ptr(pb) || !is_device_ptr(inter) || !is_device_ptr(out)) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)std::min<long long>((n_pairs + 255) / 256, 8LL * ctx->sm_count);
    k_contains<<<grid, 256, 0, st>>>(pa, pb, inter, A->area, B->area, A->n, B->n, n_pairs, out);
    SCCG_LAUNCHED(ctx, "k_contains");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_touches(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa, const int32_t* pb,
                 int64_t n_pairs, uint8_t* out, void* stream)
{
    if (!ctx || n_pairs < 0) return SCCG_EINVAL;
    if (check_prepared(A) || check_prepared(B)) return SCCG_EINVAL;
    if (n_pairs == 0) return SCCG_OK;
    if (!is_device_ptr(pa) || !is_device_ptr(pb) || !is_device_ptr(out)) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)grid_for(ctx, n_pairs, 8, 16);
    k_touches<<<grid, 256, 0, st>>>(pa, pb, n_pairs, A->n, B->n, A->off, A->xy, B->off, B->xy, out);
    SCCG_LAUNCHED(ctx, "k_touches");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_gather_pairs(sccg_ctx* ctx, const int32_t* src_pa, const int32_t* src_pb, const int64_t* seg_src,
                      const int64_t* seg_dst, int32_t n_segments, int32_t* dst_pa, int32_t* dst_pb, void* stream)
{
    if (!ctx || n_segments < 0) return SCCG_EINVAL;
    if (n_segments == 0) return SCCG_OK;
    if (!is_device_ptr(src_pa) || !is_device_ptr(src_pb) || !is_device_ptr(seg_src) || !is_device_ptr(seg_dst) ||
        !is_device_ptr(dst_pa) || !is_device_ptr(dst_pb))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)std::min<long long>(n_segments, 8LL * ctx->sm_count);
    k_gather_pairs<<<grid, 256, 0, st>>>(src_pa, src_pb, seg_src, seg_dst, n_segments, dst_pa, dst_pb);
    SCCG_LAUNCHED(ctx, "k_gather_pairs");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_jaccard_segments(sccg_ctx* ctx, const int64_t* inter, const int64_t* uni, const int64_t* seg_off,
                          int32_t n_segments, sccg_jaccard_result* out, void* stream)
{
    static_assert(sizeof(JaccardOut) == sizeof(sccg_jaccard_result), "layout");
    if (!ctx || !out || n_segments < 0) return SCCG_EINVAL;
    if (n_segments == 0) return SCCG_OK;
    if (!is_device_ptr(inter) || !is_device_ptr(uni) || !is_device_ptr(seg_off) || !is_device_ptr(out))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const unsigned grid = (unsigned)std::min<long long>(n_segments, 8LL * ctx->sm_count);
    k_jaccard_segments<<<grid, 256, 0, st>>>(inter, uni, seg_off, n_segments, reinterpret_cast<JaccardOut*>(out));
    SCCG_LAUNCHED(ctx, "k_jaccard_segments");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_launch_count(const sccg_ctx* ctx, uint64_t* out)
{
    if (!ctx || !out) return SCCG_EINVAL;
    *out = ctx->launches;
    return SCCG_OK;
}

int sccg_jaccard(sccg_ctx* ctx, const int64_t* inter, const int64_t* uni, int64_t n_pairs,
                 sccg_jaccard_result* out, void* stream)
{
    static_assert(sizeof(JaccardOut) == sizeof(sccg_jaccard_result), "layout");
    if (!ctx || !out || n_pairs < 0) return SCCG_EINVAL;
    if (n_pairs >= kJaccardMaxPairs) return SCCG_ERANGE;
    if (n_pairs > 0 && (!is_device_ptr(inter) || !is_device_ptr(uni))) return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const bool dev_out = is_device_ptr(out);
    int r = ws_reserve(ctx, jaccard_scratch(ctx, n_pairs));
    if (r) return r;
    Carve cv(ctx->ws);
    cv.take<JPart>(jaccard_parts(ctx, n_pairs));
    JaccardOut* res = dev_out ? reinterpret_cast<JaccardOut*>(out) : cv.take<JaccardOut>(1);
    r = jaccard_launch(ctx, inter, uni, n_pairs, res, st);
    if (r) return r;
    if (!dev_out) {
        r = small_copy(ctx, ctx->pinned_dev, res, sizeof(JaccardOut), st);
        if (r) return r;
        SCCG_CUDA(ctx, cudaStreamSynchronize(st));
        memcpy(out, ctx->pinned, sizeof(JaccardOut));
    }
    return SCCG_OK;
}

int sccg_copy(sccg_ctx* ctx, void* dst, const void* src, int64_t bytes, void* stream)
{
    if (!ctx || bytes < 0) return SCCG_EINVAL;
    if (bytes == 0) return SCCG_OK;
    if ((bytes & 3) || (reinterpret_cast<uintptr_t>(dst) & 3) || (reinterpret_cast<uintptr_t>(src) & 3))
        return SCCG_EINVAL;
    DeviceGuard g(ctx->device);
    // bind the device's context to this host thread before the pointer queries: a thread that has
    // made no other CUDA call yet has none current, and the queries then find no device address
    if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "sccg_copy");
    char* d = static_cast<char*>(device_view(dst, ctx->device));
    const char* s = static_cast<const char*>(device_view(src, ctx->device));
    if (!d || !s) {
        snprintf(ctx->last_err, sizeof ctx->last_err,
                 "sccg_copy: %s is neither device memory of this device nor page-locked host memory",
                 d ? "src" : "dst");
        return SCCG_EINVAL;
    }
    if (d < s + bytes && s < d + bytes) return SCCG_EINVAL;       // overlapping ranges
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the widest unit both addresses are aligned to; the remaining bytes (a multiple of 4) as words
    const uintptr_t mis = reinterpret_cast<uintptr_t>(d) | reinterpret_cast<uintptr_t>(s);
    const int unit = (mis & 15) == 0 ? 16 : (mis & 7) == 0 ? 8 : 4;
    const long long n = bytes / unit;
    const int tail = (int)((bytes - n * unit) / 4);
    const long long per_cta = 512LL * 4 * unit;        // one pass of four loads per thread
    const unsigned grid = (unsigned)std::max<long long>(1, std::min<long long>(kCopyCTAs, (n * unit + per_cta - 1) / per_cta));
    const uint32_t* st_src = reinterpret_cast<const uint32_t*>(s + n * unit);
    uint32_t* st_dst = reinterpret_cast<uint32_t*>(d + n * unit);
    if (unit == 16)
        k_copy_units<int4><<<grid, 512, 0, st>>>(reinterpret_cast<const int4*>(s), reinterpret_cast<int4*>(d), n,
                                                 st_src, st_dst, tail);
    else if (unit == 8)
        k_copy_units<int2><<<grid, 512, 0, st>>>(reinterpret_cast<const int2*>(s), reinterpret_cast<int2*>(d), n,
                                                 st_src, st_dst, tail);
    else
        k_copy_units<uint32_t><<<grid, 512, 0, st>>>(reinterpret_cast<const uint32_t*>(s), reinterpret_cast<uint32_t*>(d),
                                                     n, st_src, st_dst, tail);
    SCCG_LAUNCHED(ctx, "k_copy_units");
    ctx->launches += 1;
    return SCCG_OK;
}

int sccg_alu_probe(int device, int32_t iters, double* ms, double* lane_ops)
{
    if (iters <= 0 || !ms || !lane_ops) return SCCG_EINVAL;
    int n_dev = 0;
    if (cudaGetDeviceCount(&n_dev) != cudaSuccess || device < 0 || device >= n_dev) {
        cudaGetLastError();
        return SCCG_EINVAL;
    }
    DeviceGuard g(device);
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) return SCCG_ECUDA;
    const unsigned grid = (unsigned)sms * 8u;         // 8 CTAs of 256 threads: 64 warps per SM
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    uint32_t* sink = nullptr;
    int r = SCCG_OK;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess || cudaMalloc(&sink, sizeof(uint32_t)) != cudaSuccess) {
        r = SCCG_ECUDA;
    }
    if (!r) {
        k_alu_probe<<<grid, 256, 0, st>>>(std::max(1, iters / 16), 0x9E3779B9u, sink);   // warm-up
        cudaEventRecord(e0, st);
        k_alu_probe<<<grid, 256, 0, st>>>(iters, 0x9E3779B9u, sink);
        cudaEventRecord(e1, st);
        float t = 0.0f;
        if (cudaGetLastError() != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess) {
            r = SCCG_ECUDA;
        } else {
            *ms = (double)t;
            *lane_ops = (double)grid * 256.0 * (double)iters * (double)kAluPerIter;
        }
    }
    cudaGetLastError();
    if (sink) cudaFree(sink);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    return r;
}

int sccg_jaccard_static(const int64_t* inter, const int64_t* uni, int64_t n_pairs, sccg_jaccard_result* out,
                        void* stream)
{
    static_assert(sizeof(JaccardOut) == sizeof(sccg_jaccard_result), "layout");
    if (n_pairs < 0 || !out) return SCCG_EINVAL;
    if (n_pairs > kStaticMaxPairs) return SCCG_ERANGE;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return SCCG_ECUDA;
    }
    if (!is_device_ptr_on(out, dev)) return SCCG_EINVAL;
    if (n_pairs > 0 && (!is_device_ptr_on(inter, dev) || !is_device_ptr_on(uni, dev))) return SCCG_EINVAL;
    JPart* parts = nullptr;
    int r = static_parts_address(&parts);
    if (r) return r;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const int nparts = (int)std::max(1LL, (n_pairs + kStaticChunk - 1) / kStaticChunk);
    k_jaccard_partial_chunked<<<nparts, 256, 0, st>>>(inter, uni, n_pairs, kStaticChunk, parts);
    k_jaccard_final<<<1, 256, 0, st>>>(parts, nparts, n_pairs, reinterpret_cast<JaccardOut*>(out));
    if (cudaGetLastError() != cudaSuccess) return SCCG_ECUDA;
    return SCCG_OK;
}

}  // extern "C"
