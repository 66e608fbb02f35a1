/*
 * sccg.h - C ABI of the GB300 (sm_103a) spatial cross-comparison library.
 *
 * The library computes, for two sets of integer polygons segmented from the same image (the two
 * "result sets" of Sec. 2.1 of Wang et al., "Accelerating Pathology Image Data Cross-Comparison on
 * CPU-GPU Hybrid Systems"), the exact pixel areas of intersection and union of every pair of
 * polygons whose bounding boxes overlap, and reduces them to Jaccard similarities.
 *
 * Pixel model (Sec. 3.1, Fig. 4a/4b). Pixel (x, y) is the unit square [x, x+1) x [y, y+1). It belongs
 * to polygon p when a ray cast from its centre (x + 1/2, y + 1/2) towards +x crosses p's boundary an
 * odd number of times. An edge whose x at the ray's row equals the centre's x exactly (the centre
 * lies on that edge) is not counted. ||p|| is the number of pixels belonging to p; ||p n q|| and
 * ||p u q|| the numbers belonging to both and to either. Areas are exact int64 counts.
 *
 * Conventions for every call:
 *   - Array arguments are DEVICE pointers owned by the caller (unless a parameter says "host").
 *     The library never frees caller memory.
 *   - Calls are enqueued on the given CUDA stream (a cudaStream_t passed as void*; NULL is the
 *     legacy default stream). Outputs are valid once the stream has reached the call, except
 *     where a call is documented as synchronous.
 *   - Every call returns an sccg_status; 0 is success. No C++ exception crosses the ABI.
 *   - Scratch memory comes from the context (allocated on first need and grown on demand; growing
 *     synchronises the device). One context must not be used from two host threads at once.
 *   - Coordinates must satisfy |x|, |y| <= 2^28 and every polygon's bounding box must be at most
 *     16384 pixels wide and high: all GPU arithmetic is exact in int32 under these bounds.
 *     sccg_prepare checks them (SCCG_ERANGE).
 */
#ifndef SCCG_H
#define SCCG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ------------------------------------------------------------------------------------------- */
/* status codes                                                                                 */
/* ------------------------------------------------------------------------------------------- */
typedef enum sccg_status {
    SCCG_OK = 0,
    SCCG_EINVAL = 1,     /* bad argument: NULL or host pointer where device memory is required,
                            negative size, polygon with fewer than 3 vertices, tiles not sorted */
    SCCG_ERANGE = 2,     /* coordinate beyond +-2^28 or polygon bounding box wider/higher than 16384 */
    SCCG_ECAPACITY = 3,  /* output array too small; the required count is still reported */
    SCCG_ENOMEM = 4,     /* scratch allocation failed */
    SCCG_ECUDA = 5,      /* a CUDA runtime call or kernel launch failed (see sccg_last_error) */
    SCCG_ETIMEOUT = 6,   /* a bounded device-side wait gave up; the kernel returned cleanly */
    SCCG_ENOTSUP = 7     /* operation not supported by this build or device */
} sccg_status;

/* Short description of a status code (static string). */
const char* sccg_status_str(int status);

/* ------------------------------------------------------------------------------------------- */
/* context                                                                                      */
/* ------------------------------------------------------------------------------------------- */
typedef struct sccg_ctx sccg_ctx;

/* Tunable parameters (Sec. 3.4: pixelization threshold T; threads per pair; the persistent form's
 * work split). All have defaults; sccg_ctx_set_param changes one by name. */
typedef struct sccg_params {
    int32_t T;               /* a box is pixelized once it holds fewer than T pixels (Sec. 3.2) */
    int32_t warps_per_cta;   /* warps per CTA in the pair-area kernels (one pair per warp) */
    int32_t split_pixels;    /* persistent form: a pair's window is cut into work items of at
                                most about this many pixels (heavy pairs spread across warps) */
    int32_t ctas_per_sm;     /* persistent form: resident CTAs per SM (0 = occupancy maximum) */
    int32_t area_method;     /* how sccg_prepare counts ||p||: SCCG_AREA_ROWS (default),
                                SCCG_AREA_PIXELBOX (same exact pixel count) or SCCG_AREA_SHOELACE
                                (rectilinear simple sets: the closed form) */
    int32_t leaf_words;      /* 1 (default): a leaf window (fewer than T pixels) is pixelized from
                                per-row parity words, each edge flipping the pixels left of its
                                crossing; 0: as 32-pixel row strips tested against every edge (the
                                per-pixel test of Sec. 3.1). Same results. */
    int32_t pair_lanes;      /* threads per pair in the persistent form's leaf path (items of at most
                                64 x 64 pixels): 32 (default) one warp per item; 1: pairs whose window
                                is at most 32 x 32 pixels with at most 64 edges in both rings are done
                                one lane per pair (beside the warp path for the others). Same results. */
    int32_t area_T;          /* sccg_prepare (ROWS and SHOELACE methods): a polygon whose bounding box
                                holds fewer than area_T pixels is counted as one leaf of streamed
                                parity words, a larger one by rows (default 65536). Same results. */
    int32_t rasters;         /* 1 (default): the pair-area calls use the sets' pixel rasters when both
                                sets have them (see sccg_polyset.raster); 0: they pixelize every pair's
                                window as without rasters. Same results. */
    int32_t raster_heavy;    /* pair areas from rasters, persistent form: a pair whose window has more
                                than raster_heavy (row, 32-pixel word) units is done by a whole CTA
                                instead of one warp (default 1024; -1: every pair by one warp). */
    int32_t raster_lanes;    /* pair areas from rasters: threads per (light) pair, 8, 16 or 32
                                (default; a warp works on 32 / raster_lanes pairs at a time), or 1:
                                a pair whose window is at most 64 x 64 pixels by one lane, the others
                                by the warp. Same results. */
} sccg_params;

/* sccg_prepare's method for ||p||. ROWS: per pixel row, the crossing positions of the edges that
 * straddle it (sorted) delimit the inside pixels, so cost follows the edges per row (the exact
 * pixel-count counterpart of the shoelace area the paper uses, Sec. 3.2). PIXELBOX: Algorithm 1
 * applied to the polygon alone. SHOELACE: for sets the caller flags as rectilinear and simple (the
 * paper's raster-boundary polygons, Sec. 3.1, Fig. 3): a polygon whose edges are all axis-parallel
 * (checked on the device) gets |shoelace area| (Sec. 3.2, POLYAREA), which equals its pixel count
 * when the ring is simple (not checked: the caller's flag vouches for it); any other polygon is
 * counted as with ROWS. */
enum { SCCG_AREA_ROWS = 0, SCCG_AREA_PIXELBOX = 1, SCCG_AREA_SHOELACE = 2 };

/* Create a context on CUDA device `device`. params_json may be NULL or a flat JSON object with any
 * of the sccg_params field names, e.g. {"T": 1024, "warps_per_cta": 8}. */
int sccg_ctx_create(int device, const char* params_json, sccg_ctx** out);
int sccg_ctx_destroy(sccg_ctx* ctx);
int sccg_ctx_set_param(sccg_ctx* ctx, const char* name, int64_t value);
int sccg_ctx_get_params(const sccg_ctx* ctx, sccg_params* out /* host */);
/* Grow the context's scratch now so that sccg_pair_areas (PERSISTENT), sccg_batch_run and
 * sccg_jaccard on up to max_pairs pairs allocate nothing later (growing synchronises the device; a
 * serving loop does it once at start-up). SCCG_ERANGE for max_pairs >= 2^43. */
int sccg_ctx_reserve(sccg_ctx* ctx, int64_t max_pairs);
/* Text of the last CUDA error seen by this context ("" if none). */
const char* sccg_last_error(const sccg_ctx* ctx);

/* ------------------------------------------------------------------------------------------- */
/* polygon sets                                                                                 */
/* ------------------------------------------------------------------------------------------- */
/* One result set in CSR form. Polygon i has vertices off[i] .. off[i+1]-1; vertex v is
 * (xy[2v], xy[2v+1]); the ring closes implicitly from the last vertex back to the first. Polygons
 * are grouped by image tile (Sec. 2.1: one polygon file per tile): tile[] is non-decreasing. */
typedef struct sccg_polyset {
    int64_t n;              /* number of polygons (>= 0) */
    const int64_t* off;     /* device, [n+1], off[0] = 0, non-decreasing */
    const int32_t* xy;      /* device, [2*off[n]], 8-byte aligned */
    const int32_t* tile;    /* device, [n], >= 0, non-decreasing; NULL = every polygon in tile 0 */
    int32_t* mbr;           /* device, [4n], written by sccg_prepare: min x, min y, max x, max y */
    int64_t* area;          /* device, [n], written by sccg_prepare: ||p|| */
    /* host-side summary written by sccg_prepare */
    int32_t max_nv;         /* largest vertex count */
    int32_t max_extent;     /* largest bounding-box width or height */
    int32_t n_tiles;        /* largest tile id + 1 */
    int32_t reserved;       /* set by sccg_prepare once the set is valid; do not modify */
    int64_t band_bytes;     /* written by sccg_prepare: device bytes sccg_build_bands needs for the
                               set's band index (0: no polygon has 1024 or more vertices) */
    const void* bands;      /* device, optional: the band index written by sccg_build_bands, or
                               NULL (then every work item reads its polygons' whole rings) */
    void* raster;           /* device, optional (NULL: none): caller-owned buffer of raster_cap bytes,
                               16-byte aligned, kept alive and unmodified while the set is used, into
                               which sccg_prepare writes the set's pixel rasters: polygon i's window
                               of W x H pixels (its MBR) as H rows of ceil(W / 32) uint32 words, bit b
                               of word k of row r set iff pixel (minx + 32 k + b, miny + r) belongs to
                               the polygon. Layout: int64 word offsets [n + 1] padded to 16 bytes
                               (polygon i's words start at word off[i]; off[n] is the total), then
                               the words: a slot of 128 words per polygon (polygon i's at word 128 i,
                               holding its raster when its window is at most 64 x 64 pixels), then
                               the rasters of the larger windows, in an order the call chooses. */
    int64_t raster_cap;     /* bytes available at raster */
    int64_t raster_bytes;   /* written by sccg_prepare when raster != NULL: bytes the rasters take
                               (offsets and words), whether they fitted or not */
    int32_t raster_ok;      /* written by sccg_prepare: 1 when the rasters were written (raster_bytes
                               <= raster_cap); the pair-area calls then use them */
    int32_t raster_pad;
} sccg_polyset;

/* Step 1 of the path: per-polygon bounding box (MBR) and pixel area ||p|| (Sec. 3.2 computes ||p||
 * with the shoelace formula for the paper's rectilinear polygons; here ||p|| is the pixel count
 * itself, which equals the shoelace area on pixel-aligned rectilinear polygons and is the value
 * that makes ||p u q|| = ||p|| + ||q|| - ||p n q|| exact for every polygon).
 * Validates the set (>= 3 vertices, coordinate bounds, tile order) and fills the host summary
 * fields; SYNCHRONISES the stream once to read the validation result back. With the default
 * area method, polygons of 1024 or more vertices get their areas after that synchronisation, from a
 * temporary band index in context scratch (kernels queued on the stream; the areas are ready when
 * the stream reaches them).
 * Returns SCCG_EINVAL or SCCG_ERANGE for invalid sets (mbr/area contents then unspecified). */
int sccg_prepare(sccg_ctx* ctx, sccg_polyset* s, void* stream);
/* With s->raster set, sccg_prepare also writes the set's pixel rasters (Sec. 3.1's pixel membership,
 * decided once per polygon and kept in device memory): each polygon is pixelized once and its ||p||
 * counted from its raster, the windows of at most 64 x 64 pixels into their slots in the pass that
 * finds the MBRs, the larger ones after the synchronisation, once their sizes are known. A pair's
 * ||p n q|| is then the number of set bits of the AND of the two rasters over the pair's window
 * (sccg_pair_areas and the calls built on it, except SCCG_MODE_NOSEP), with the same results. The
 * area method does not apply to a set with rasters. When the rasters do not fit (raster_bytes >
 * raster_cap), raster_ok is 0 and the set is prepared as without rasters (the buffer's contents are
 * then unspecified); sccg_raster_bytes gives the size beforehand. */

/* Bytes the pixel rasters of set s take (offsets and words), for sizing s->raster. Computes and
 * writes the set's MBRs (s->mbr) on the way, validates the set as sccg_prepare does and SYNCHRONISES
 * the stream once. bytes: host out. */
int sccg_raster_bytes(sccg_ctx* ctx, sccg_polyset* s, int64_t* bytes, void* stream);

/* sccg_prepare for n_sets sets (1..64) at once: their kernels are launched back to back and the
 * stream is synchronised once. Every set's summary is filled in; a set that fails validation is not
 * marked prepared, and the call returns the first failure's status (SCCG_OK if none). */
int sccg_prepare_sets(sccg_ctx* ctx, sccg_polyset* sets, int n_sets, void* stream);

/* Band index of the set's polygons with 1024 or more vertices (large tissue regions): each such
 * polygon's rows are cut into 32-row bands and every band lists the edges whose y-range meets it,
 * so a pair-area work item reads only the edges near its window instead of the whole ring (the
 * sampling boxes of Sec. 3.2 only ever test edges that can meet them; this finds those edges
 * without scanning every vertex). Optional: results are identical with and without it.
 * buf: caller-owned device memory of at least s->band_bytes bytes, 16-byte aligned, kept alive and
 * unmodified while the set is used; on success s->bands = buf. s must have been prepared.
 * Asynchronous on `stream`. Returns SCCG_ECAPACITY when bytes < s->band_bytes (s->bands unchanged);
 * with s->band_bytes == 0 it sets s->bands = NULL and launches nothing. */
int sccg_build_bands(sccg_ctx* ctx, sccg_polyset* s, void* buf, int64_t bytes, void* stream);

/* ------------------------------------------------------------------------------------------- */
/* the hot path                                                                                 */
/* ------------------------------------------------------------------------------------------- */

/* Filter stage (Sec. 4.1 stage 3; the && operator of Fig. 1b): every pair (a, b) with
 * tile_A[a] == tile_B[b] whose closed MBRs overlap (ax0 <= bx1 && bx0 <= ax1 && ay0 <= by1 &&
 * by0 <= ay1), written to pa[k], pb[k] in ascending (a, b) order. Both sets must be prepared.
 *   capacity        entries available in pa/pb
 *   n_pairs         HOST out: total number of pairs (also when it exceeds capacity)
 *   tile_pair_off   out [n_tiles + 1], device or host memory (may be NULL): first pair index of
 *                   each tile, where
 *                   n_tiles = max(A.n_tiles, B.n_tiles); tile t owns pairs
 *                   tile_pair_off[t] .. tile_pair_off[t+1]-1.
 * SYNCHRONISES the stream once (to return the count). SCCG_ECAPACITY if the pairs do not fit
 * (nothing beyond capacity is written). */
int sccg_candidate_pairs(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B,
                         int32_t* pa, int32_t* pb, int64_t capacity, int64_t* n_pairs,
                         int64_t* tile_pair_off, void* stream);

/* Aggregator stage (Sec. 3, Algorithm 1): for each pair k, inter[k] = ||p n q|| and
 * uni[k] = ||p|| + ||q|| - ||p n q|| (Sec. 3.2, areas of union computed indirectly), with
 * p = A polygon pa[k] and q = B polygon pb[k]. A pair whose indices fall outside [0, A.n) or
 * [0, B.n) is not evaluated: its inter and uni are set to -1. ||p n q|| is found by recursive sampling-box
 * subdivision of the pair's window MBR(p) n MBR(q) (Sec. 3.2): boxes entirely inside both polygons
 * add their pixel count, boxes outside either add nothing, and boxes still mixed once they hold
 * fewer than T pixels are pixelized (Sec. 3.1). Both sets must be prepared. Asynchronous.
 *   mode SCCG_MODE_PLAIN       one warp per pair, grid-stride over the n_pairs given (the caller
 *                              launches once per tile for the one-launch-per-tile form)
 *   mode SCCG_MODE_PERSISTENT  resident CTAs pull work items from a device queue; pairs with large
 *                              windows are cut into several items whose partial counts are added
 *                              with 64-bit atomics (Sec. 4.1's batching, on the device)
 *   mode SCCG_MODE_NOSEP       the PixelBox-NoSep variant of Sec. 5.2 (Fig. 8), for comparison: as
 *                              PLAIN, but uni[k] is counted directly by subdivision of the bounding
 *                              box of MBR(p) u MBR(q) instead of from the areas. Same results.
 *                              SCCG_ERANGE if either set has a polygon wider or taller than 8192 px.
 * A pixelization-only run (PixelOnly of Sec. 5.2) is PLAIN with T above every window (T = 2^28). */
#define SCCG_MODE_PLAIN 0
#define SCCG_MODE_PERSISTENT 1
#define SCCG_MODE_NOSEP 2
int sccg_pair_areas(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B,
                    const int32_t* pa, const int32_t* pb, int64_t n_pairs,
                    int64_t* inter, int64_t* uni, int mode, void* stream);

/* The one-launch-per-tile form of the aggregator (Sec. 4.1: a task is one image tile): the same
 * result as sccg_pair_areas in PLAIN mode, with one kernel launch per tile that has pairs.
 *   tile_pair_off  HOST [n_tiles + 1]: tile t owns pairs tile_pair_off[t] .. tile_pair_off[t+1]-1
 *                  (as written by sccg_candidate_pairs); must start at 0 and be non-decreasing.
 * The launches are spread round-robin over 8 internal streams forked from `stream` (so independent
 * tiles may run concurrently) and joined back into it before the call returns. Asynchronous. */
int sccg_pair_areas_tiles(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B,
                          const int32_t* pa, const int32_t* pb, const int64_t* tile_pair_off,
                          int32_t n_tiles, int64_t* inter, int64_t* uni, void* stream);

/* Number of kernels this context has launched so far (all calls). */
int sccg_launch_count(const sccg_ctx* ctx, uint64_t* out /* host */);

/* Jaccard reductions of Sec. 2.1 over the pairs with inter > 0 (Sec. 4.1: pairs that do not
 * actually intersect are not considered):
 *   J  = sum inter / sum union                 (double(sum_inter) / double(sum_union))
 *   J' = (1/n_nonzero) sum inter_k / union_k   (Eq. 1)
 * Each ratio is the IEEE double quotient; the ratios are summed exactly in 128-bit fixed point and
 * rounded once to the nearest double, then divided by n_nonzero, so J' does not depend on the
 * summation order. Both are 0 when no pair intersects. The fixed-point sum is exact for fewer than
 * 2^43 pairs: larger n_pairs return SCCG_ERANGE (here and in sccg_batch_run; a segment of
 * sccg_jaccard_segments cannot hold that many pairs in device memory).
 * `out` may be a host pointer (the call then SYNCHRONISES the stream) or a device pointer (the
 * call stays asynchronous and writes the struct on the stream). */
typedef struct sccg_jaccard_result {
    int64_t sum_inter;
    int64_t sum_union;
    int64_t n_nonzero;
    int64_t n_pairs;
    double J;
    double Jprime;
} sccg_jaccard_result;
int sccg_jaccard(sccg_ctx* ctx, const int64_t* inter, const int64_t* uni, int64_t n_pairs,
                 sccg_jaccard_result* out, void* stream);

/* Batched form (Sec. 4.1: the aggregator groups many tile tasks into one GPU batch; the batched step):
 * the persistent pair areas and unions of sccg_pair_areas(PERSISTENT) followed by the Jaccard
 * reductions into the DEVICE result `out`, replayed as one CUDA graph. The graph is captured on the
 * first call and re-captured only when the pointers, the pair count or the parameters change, so
 * repeated calls on the same buffers cost one graph launch. Asynchronous. Scratch is sized before
 * capture; the context must not be used for other calls while the graph may be running. */
int sccg_batch_run(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B,
                   const int32_t* pa, const int32_t* pb, int64_t n_pairs,
                   int64_t* inter, int64_t* uni, sccg_jaccard_result* out, void* stream);


/* Other spatial operators through the same machinery (Sec. 3.4, "Implications of PixelBox to other
 * spatial operators"; device arrays, asynchronous, both sets prepared):
 * sccg_contains: ST_Contains from the pixel areas, as the paper states it: out[k] bit 0 is set when
 *   the A polygon contains the B polygon (inter[k] = ||q|| > 0), bit 1 when the B polygon contains
 *   the A polygon (inter[k] = ||p|| > 0); inter from sccg_pair_areas. 0xff for invalid pairs.
 * sccg_touches: ST_Touches by the paper's rule, in exact integer geometry on the vertex rings: 1 when
 *   no edge of one crosses an edge of the other (segment interiors crossing at one point), no vertex
 *   of one lies strictly within the other (even-odd, not on its boundary) and some vertex of one lies
 *   on an edge of the other; else 0 (0xff for invalid pairs). The rule also reports a touch for
 *   polygons whose interiors overlap without any vertex strictly inside or any proper crossing
 *   (e.g. one inside the other along shared edges). O(n_p n_q) per pair, one warp per pair. */
int sccg_contains(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa, const int32_t* pb,
                  const int64_t* inter, int64_t n_pairs, uint8_t* out, void* stream);
int sccg_touches(sccg_ctx* ctx, const sccg_polyset* A, const sccg_polyset* B, const int32_t* pa, const int32_t* pb,
                 int64_t n_pairs, uint8_t* out, void* stream);

/* Add base_a to pa[k] and base_b to pb[k] for k < n_pairs: turns the candidate pairs of a chunk of
 * tiles (polygon indices local to the chunk's sub-sets) into indices of the whole sets, for a
 * pipelined front end that copies and compares chunks in turn (Sec. 4.1, Fig. 6; the paper has no
 * such call). Bases in [0, 2^31); the caller keeps base + local index below 2^31. Asynchronous. */
int sccg_rebase_pairs(sccg_ctx* ctx, int32_t* pa, int32_t* pb, int64_t n_pairs, int64_t base_a, int64_t base_b,
                      void* stream);

/* Allocation-free variant of sccg_jaccard (the paper has no counterpart; this is a library
 * service). Same results as sccg_jaccard, but it needs no context and allocates nothing: its scratch
 * (4096 partial-sum slots, 160 KB) is a fixed array in device memory that every GPU loading this
 * library keeps until the process exits. It is meant for callers that must not allocate device
 * memory: plugins inside a host application that owns all device memory through its own pool or
 * budget (a cudaMalloc of theirs would go around it, or fail because the pool holds the device),
 * deployments that forbid allocation after start-up, and latency-critical loops where
 * cudaMalloc/cudaFree would synchronise the device.
 *   inter, uni  device, [n_pairs] (as written by sccg_pair_areas)
 *   out         DEVICE pointer to one sccg_jaccard_result, written asynchronously on `stream`
 *   n_pairs     at most 268,435,456 (4096 slots x 65,536 pairs); larger counts return SCCG_ERANGE
 * Every call looks up the array's device address in the current context (a context the caller
 * created with the driver API has its own copy of the array); the first call in a context also loads
 * the library's kernels there, so make that first call before any stream capture. inter, uni, out
 * and `stream` must belong to the current device. All calls share the one array and leave their
 * partial sums in it; each call writes every slot it reads before reading it, so nothing needs
 * clearing, but two calls whose work overlaps on the GPU (different streams, or different host
 * threads) race on the array and must be serialised by the caller. Returns SCCG_EINVAL for host
 * pointers, pointers on another device or n_pairs < 0. */
int sccg_jaccard_static(const int64_t* inter, const int64_t* uni, int64_t n_pairs,
                        sccg_jaccard_result* out, void* stream);

/* Batch assembly for the serving loop (Sec. 4.1: the aggregator groups tasks into GPU batches):
 * copies n_segments slices of the pair arrays, slice s = src[seg_src[s] .. seg_src[s] + len_s),
 * len_s = seg_dst[s+1] - seg_dst[s], to dst[seg_dst[s] ..). All pointers are device memory;
 * seg_dst has n_segments + 1 entries. Asynchronous. */
int sccg_gather_pairs(sccg_ctx* ctx, const int32_t* src_pa, const int32_t* src_pb,
                      const int64_t* seg_src, const int64_t* seg_dst, int32_t n_segments,
                      int32_t* dst_pa, int32_t* dst_pb, void* stream);

/* Per-segment Jaccard reductions (Sec. 2.1, Eq. 1, with the same exact rounding as sccg_jaccard):
 * segment s covers pairs seg_off[s] .. seg_off[s+1]-1 (one job of a serving batch, or one tile);
 * out is a DEVICE array of n_segments results. Asynchronous. */
int sccg_jaccard_segments(sccg_ctx* ctx, const int64_t* inter, const int64_t* uni,
                          const int64_t* seg_off, int32_t n_segments,
                          sccg_jaccard_result* out, void* stream);

/* Copy of `bytes` bytes from src to dst by the SMs instead of the copy engines, for the pipelined
 * front end (Sec. 4.1, Fig. 6: each chunk's polygons move host -> device while the previous chunk is
 * compared). Each of dst and src is device memory of the context's device or page-locked host
 * memory mapped into the device's address space (cudaHostAlloc / cudaHostRegister), which the
 * kernel reads or writes directly over the host link; 16 CTAs of 512 threads keep that link full
 * while leaving the other SMs to the comparison kernels. bytes and both addresses must be multiples
 * of 4 and the ranges must not overlap. Asynchronous on `stream`. Returns SCCG_EINVAL for pageable
 * or unknown memory, another device's memory, misalignment or overlap (nothing is launched). */
int sccg_copy(sccg_ctx* ctx, void* dst, const void* src, int64_t bytes, void* stream);

/* ------------------------------------------------------------------------------------------- */
/* measurement                                                                                  */
/* ------------------------------------------------------------------------------------------- */
/* Integer ALU issue rate of CUDA device `device`, the denominator against which the pair-area and
 * prepare kernels' integer work is reported (the paper has no counterpart; Sec. 3.3 and Sec. 5.3
 * argue the method is bound by the per-pixel and per-box position tests). Runs one kernel of 8 CTAs of
 * 256 threads per SM, each thread `iters` iterations of 24 independent-chain int32 operations
 * (multiply-add, three-input XOR, three-input add: one integer-unit instruction each), after a short
 * warm-up, on a private stream timed by CUDA events. ms (host): the kernel's time; lane_ops (host):
 * the int32 operations it executed (lane_ops / ms is the rate). Synchronous; allocates a few bytes. */
int sccg_alu_probe(int device, int32_t iters, double* ms, double* lane_ops);

/* ------------------------------------------------------------------------------------------- */
/* work accounting                                                                              */
/* ------------------------------------------------------------------------------------------- */
/* With sccg_ctx_set_param(ctx, "count_work", 1) the prepare and pair-area kernels run an
 * instrumented build that counts the work the method performs; the counts accumulate in the
 * context until read. out12 (host, 12 entries): [0] (32-pixel row strip, edge) evaluations of the
 * full strip test, [1] (pixel, edge) point-in-polygon tests inside those strips, [2] (sampling box,
 * edge) classifications, [3] sampling boxes classified, [4] (edge, row) crossings XORed into leaf
 * parity words, [5] (row, 32-pixel word) parity words reduced, [6] (edge, row) crossing values of
 * the by-rows area (and crossings drawn into the difference rows of large rasters), [7]
 * crossing-value comparisons ranking them, [8] (pixel, polygon) memberships decided one pixel at a
 * time (leaves), [9] pixels of the windows counted, [10] raster words written, [11] (row, 32-pixel
 * word) ANDs of two rasters over pair windows. Synchronous. reset != 0 zeroes the counters. */
int sccg_work_counters(sccg_ctx* ctx, uint64_t* out12, int reset);

#ifdef __cplusplus
}
#endif

#endif /* SCCG_H */
