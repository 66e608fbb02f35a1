/*
 * CPU oracle for the PixelBox cross-comparison quantities (test infrastructure only).
 *
 * This file is the plain, slow, obviously correct definition of what the GPU path computes. It is
 * used only by the tests, by the smoke check and by the CPU-baseline leg of the benchmark; no
 * product code links it. It shares no code, header or table with the CUDA library.
 *
 * Definitions (Sec. 3.1 of the paper, with the exact tie rule written out):
 *   - Pixel (x, y) is the unit square [x, x+1) x [y, y+1); its centre is (x + 1/2, y + 1/2).
 *   - A pixel belongs to polygon p when a horizontal ray cast from its centre towards +x crosses
 *     the boundary of p an odd number of times (ray casting, Sec. 3.1 and Fig. 4b; even-odd rule).
 *   - Crossing rule, in doubled coordinates (vertices (2x, 2y) are even, the centre (2x+1, 2y+1) is
 *     odd, so the ray never passes through a vertex): edge (X1,Y1)->(X2,Y2) straddles the ray row
 *     when (Y1 > Cy) != (Y2 > Cy); oriented so that Y1 < Y2, it is crossed when the edge's x at row Cy
 *     is strictly greater than Cx, i.e. (Cx - X1)*(Y2 - Y1) < (Cy - Y1)*(X2 - X1). A centre exactly
 *     on the edge does not count that edge.
 *   - ||p|| is the number of pixels belonging to p; ||p n q|| the number belonging to both and
 *     ||p u q|| the number belonging to either (Sec. 3.1, Fig. 4a). The pair functions below count
 *     intersection and union directly over every pixel of the bounding box of MBR(p) u MBR(q).
 *   - MBR(p) = [min x, max x] x [min y, max y] over p's vertices; the pixels whose centres can lie
 *     inside it are x in [min x, max x - 1], y in [min y, max y - 1].
 *   - Candidate pairs (the filter stage, Sec. 4.1, and the && operator of Fig. 1b): all (a, b) with
 *     the same tile id whose closed MBRs overlap, in ascending (a, b) order.
 *
 * A second, independent exact method (row intervals) is provided for cross-checking the brute force
 * and for checking large workloads whose brute force would take too long: for each pixel row it
 * computes, per straddling edge, the first pixel column not crossed, sorts these thresholds and
 * takes alternate intervals. It shares nothing with the brute force beyond the definition.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef int64_t i64;

/* ------------------------------------------------------------------------------------------- */
/* brute force                                                                                  */
/* ------------------------------------------------------------------------------------------- */

/* 1 when pixel (px, py) belongs to the polygon with nv vertices xy[2*i], xy[2*i+1]. */
int oracle_pixel_in_polygon(const int32_t* xy, i64 nv, i64 px, i64 py)
{
    const i64 cx = 2 * px + 1, cy = 2 * py + 1;
    int inside = 0;
    for (i64 i = 0; i < nv; ++i) {
        const i64 j = (i + 1 == nv) ? 0 : i + 1;
        i64 x1 = 2 * (i64)xy[2 * i], y1 = 2 * (i64)xy[2 * i + 1];
        i64 x2 = 2 * (i64)xy[2 * j], y2 = 2 * (i64)xy[2 * j + 1];
        if ((y1 > cy) != (y2 > cy)) {
            if (y1 > y2) { i64 t = x1; x1 = x2; x2 = t; t = y1; y1 = y2; y2 = t; }
            if ((cx - x1) * (y2 - y1) < (cy - y1) * (x2 - x1)) inside ^= 1;
        }
    }
    return inside;
}

/* MBR of one polygon: out[0..3] = min x, min y, max x, max y. */
void oracle_mbr(const int32_t* xy, i64 nv, int32_t* out)
{
    int32_t x0 = xy[0], y0 = xy[1], x1 = xy[0], y1 = xy[1];
    for (i64 i = 1; i < nv; ++i) {
        if (xy[2 * i] < x0) x0 = xy[2 * i];
        if (xy[2 * i] > x1) x1 = xy[2 * i];
        if (xy[2 * i + 1] < y0) y0 = xy[2 * i + 1];
        if (xy[2 * i + 1] > y1) y1 = xy[2 * i + 1];
    }
    out[0] = x0; out[1] = y0; out[2] = x1; out[3] = y1;
}

/* ||p||: count of pixels belonging to p over the pixel window of MBR(p). */
i64 oracle_polygon_area(const int32_t* xy, i64 nv)
{
    int32_t m[4];
    oracle_mbr(xy, nv, m);
    i64 area = 0;
    for (i64 y = m[1]; y < m[3]; ++y)
        for (i64 x = m[0]; x < m[2]; ++x)
            area += oracle_pixel_in_polygon(xy, nv, x, y);
    return area;
}

/* Membership mask of p over the pixel window of MBR(p): out[(y - min y) * W + (x - min x)] = 1 when
 * pixel (x, y) belongs to p (W = max x - min x), by the per-pixel test above. */
void oracle_polygon_mask(const int32_t* xy, i64 nv, uint8_t* out)
{
    int32_t m[4];
    oracle_mbr(xy, nv, m);
    const i64 W = (i64)m[2] - m[0];
    for (i64 y = m[1]; y < m[3]; ++y)
        for (i64 x = m[0]; x < m[2]; ++x)
            out[(y - m[1]) * W + (x - m[0])] = (uint8_t)oracle_pixel_in_polygon(xy, nv, x, y);
}

/* ||p n q|| and ||p u q||, both counted directly over the bounding box of MBR(p) u MBR(q). */
void oracle_pair(const int32_t* xp, i64 np, const int32_t* xq, i64 nq, i64* inter, i64* uni)
{
    int32_t a[4], b[4];
    oracle_mbr(xp, np, a);
    oracle_mbr(xq, nq, b);
    const i64 x0 = a[0] < b[0] ? a[0] : b[0], y0 = a[1] < b[1] ? a[1] : b[1];
    const i64 x1 = a[2] > b[2] ? a[2] : b[2], y1 = a[3] > b[3] ? a[3] : b[3];
    i64 in = 0, un = 0;
    for (i64 y = y0; y < y1; ++y)
        for (i64 x = x0; x < x1; ++x) {
            const int ip = oracle_pixel_in_polygon(xp, np, x, y);
            const int iq = oracle_pixel_in_polygon(xq, nq, x, y);
            in += ip & iq;
            un += ip | iq;
        }
    *inter = in;
    *uni = un;
}

/* ------------------------------------------------------------------------------------------- */
/* row-interval method (independent cross-check)                                               */
/* ------------------------------------------------------------------------------------------- */

static i64 ceil_div(i64 a, i64 b) /* b > 0 */
{
    i64 q = a / b, r = a % b;
    return (r != 0 && a > 0) ? q + 1 : q;
}

static int cmp_i64(const void* a, const void* b)
{
    const i64 u = *(const i64*)a, v = *(const i64*)b;
    return (u > v) - (u < v);
}

/* Pixel x of row y is crossed by edge e (straddling y) iff x < t_e(y), the first uncrossed column:
 * crossing  <=>  (2x+1-2xl)*dy < (2y+1-2yl)*dx  <=>  2x*dy < N,  N = (2y+1-2yl)*dx + (2xl-1)*dy,
 * so t_e(y) = ceil(N / (2 dy)). The pixels with an odd number of thresholds above them are the
 * union of [t1, t2), [t3, t4), ... of the sorted thresholds. Writes that list into iv (pairs) and
 * returns the number of intervals. buf must hold nv entries. */
static i64 row_intervals(const int32_t* xy, i64 nv, i64 y, i64* buf, i64* iv)
{
    i64 m = 0;
    for (i64 i = 0; i < nv; ++i) {
        const i64 j = (i + 1 == nv) ? 0 : i + 1;
        i64 xa = xy[2 * i], ya = xy[2 * i + 1], xb = xy[2 * j], yb = xy[2 * j + 1];
        if (ya == yb) continue;
        if (ya > yb) { i64 t = xa; xa = xb; xb = t; t = ya; ya = yb; yb = t; }
        if (!(ya <= y && y < yb)) continue;
        const i64 dx = xb - xa, dy = yb - ya;
        const i64 N = (2 * y + 1 - 2 * ya) * dx + (2 * xa - 1) * dy;
        buf[m++] = ceil_div(N, 2 * dy);
    }
    qsort(buf, (size_t)m, sizeof(i64), cmp_i64);
    i64 k = 0;
    for (i64 i = 0; i + 1 < m; i += 2) {
        if (buf[i + 1] > buf[i]) { iv[2 * k] = buf[i]; iv[2 * k + 1] = buf[i + 1]; ++k; }
    }
    return k;
}

static i64 overlap_len(const i64* a, i64 na, const i64* b, i64 nb)
{
    i64 i = 0, j = 0, s = 0;
    while (i < na && j < nb) {
        const i64 lo = a[2 * i] > b[2 * j] ? a[2 * i] : b[2 * j];
        const i64 hi = a[2 * i + 1] < b[2 * j + 1] ? a[2 * i + 1] : b[2 * j + 1];
        if (hi > lo) s += hi - lo;
        if (a[2 * i + 1] < b[2 * j + 1]) ++i; else ++j;
    }
    return s;
}

i64 oracle_rle_area(const int32_t* xy, i64 nv)
{
    int32_t m[4];
    oracle_mbr(xy, nv, m);
    i64* buf = (i64*)malloc(sizeof(i64) * (size_t)(nv + 1));
    i64* iv = (i64*)malloc(sizeof(i64) * (size_t)(nv + 2));
    i64 area = 0;
    for (i64 y = m[1]; y < m[3]; ++y) {
        const i64 k = row_intervals(xy, nv, y, buf, iv);
        for (i64 i = 0; i < k; ++i) area += iv[2 * i + 1] - iv[2 * i];
    }
    free(buf); free(iv);
    return area;
}

/* The membership mask of oracle_polygon_mask from the row intervals (for windows too large for the
 * brute force): the pixels of row y inside p are those of its intervals, clipped to the window. */
void oracle_rle_mask(const int32_t* xy, i64 nv, uint8_t* out)
{
    int32_t m[4];
    oracle_mbr(xy, nv, m);
    const i64 W = (i64)m[2] - m[0];
    i64* buf = (i64*)malloc(sizeof(i64) * (size_t)(nv + 1));
    i64* iv = (i64*)malloc(sizeof(i64) * (size_t)(nv + 2));
    for (i64 y = m[1]; y < m[3]; ++y) {
        uint8_t* row = out + (y - m[1]) * W;
        memset(row, 0, (size_t)W);
        const i64 k = row_intervals(xy, nv, y, buf, iv);
        for (i64 i = 0; i < k; ++i) {
            const i64 lo = iv[2 * i] > m[0] ? iv[2 * i] : m[0];
            const i64 hi = iv[2 * i + 1] < m[2] ? iv[2 * i + 1] : m[2];
            for (i64 x = lo; x < hi; ++x) row[x - m[0]] = 1;
        }
    }
    free(buf); free(iv);
}

void oracle_rle_pair(const int32_t* xp, i64 np, const int32_t* xq, i64 nq, i64* inter, i64* uni)
{
    int32_t a[4], b[4];
    oracle_mbr(xp, np, a);
    oracle_mbr(xq, nq, b);
    const i64 nmax = (np > nq ? np : nq) + 2;
    i64* buf = (i64*)malloc(sizeof(i64) * (size_t)nmax);
    i64* ivp = (i64*)malloc(sizeof(i64) * (size_t)nmax);
    i64* ivq = (i64*)malloc(sizeof(i64) * (size_t)nmax);
    const i64 y0 = a[1] < b[1] ? a[1] : b[1], y1 = a[3] > b[3] ? a[3] : b[3];
    i64 in = 0, ap = 0, aq = 0;
    for (i64 y = y0; y < y1; ++y) {
        const i64 kp = (y >= a[1] && y < a[3]) ? row_intervals(xp, np, y, buf, ivp) : 0;
        const i64 kq = (y >= b[1] && y < b[3]) ? row_intervals(xq, nq, y, buf, ivq) : 0;
        for (i64 i = 0; i < kp; ++i) ap += ivp[2 * i + 1] - ivp[2 * i];
        for (i64 i = 0; i < kq; ++i) aq += ivq[2 * i + 1] - ivq[2 * i];
        in += overlap_len(ivp, kp, ivq, kq);
    }
    free(buf); free(ivp); free(ivq);
    *inter = in;
    *uni = ap + aq - in;
}

/* ------------------------------------------------------------------------------------------- */
/* batched drivers (threads over polygons or pairs)                                            */
/* ------------------------------------------------------------------------------------------- */

typedef struct {
    const i64* off_a; const int32_t* xy_a;
    const i64* off_b; const int32_t* xy_b;
    const i64* pa; const i64* pb;      /* pair lists (NULL for per-polygon jobs) */
    i64 n;
    i64* out0; i64* out1;
    int method;                        /* 0 brute force, 1 row intervals */
    int nthreads, tid;
} job_t;

static void* pair_worker(void* arg)
{
    job_t* j = (job_t*)arg;
    for (i64 i = j->tid; i < j->n; i += j->nthreads) {
        const i64 a = j->pa[i], b = j->pb[i];
        const int32_t* xp = j->xy_a + 2 * j->off_a[a];
        const int32_t* xq = j->xy_b + 2 * j->off_b[b];
        const i64 np = j->off_a[a + 1] - j->off_a[a], nq = j->off_b[b + 1] - j->off_b[b];
        if (j->method == 0) oracle_pair(xp, np, xq, nq, &j->out0[i], &j->out1[i]);
        else oracle_rle_pair(xp, np, xq, nq, &j->out0[i], &j->out1[i]);
    }
    return NULL;
}

static void* area_worker(void* arg)
{
    job_t* j = (job_t*)arg;
    for (i64 i = j->tid; i < j->n; i += j->nthreads) {
        const int32_t* xp = j->xy_a + 2 * j->off_a[i];
        const i64 np = j->off_a[i + 1] - j->off_a[i];
        j->out0[i] = (j->method == 0) ? oracle_polygon_area(xp, np) : oracle_rle_area(xp, np);
        oracle_mbr(xp, np, (int32_t*)(j->out1) + 4 * i);
    }
    return NULL;
}

static void run_threads(job_t* proto, int nthreads, void* (*fn)(void*))
{
    if (nthreads < 1) nthreads = 1;
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * (size_t)nthreads);
    job_t* jobs = (job_t*)malloc(sizeof(job_t) * (size_t)nthreads);
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = *proto;
        jobs[t].nthreads = nthreads;
        jobs[t].tid = t;
        pthread_create(&th[t], NULL, fn, &jobs[t]);
    }
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    free(th); free(jobs);
}

/* Per-pair inter and union for pairs (pa[i], pb[i]); method 0 = brute force, 1 = row intervals. */
void oracle_pair_areas(const i64* off_a, const int32_t* xy_a, const i64* off_b, const int32_t* xy_b,
                       const i64* pa, const i64* pb, i64 n, i64* inter, i64* uni,
                       int method, int nthreads)
{
    job_t j;
    memset(&j, 0, sizeof j);
    j.off_a = off_a; j.xy_a = xy_a; j.off_b = off_b; j.xy_b = xy_b;
    j.pa = pa; j.pb = pb; j.n = n; j.out0 = inter; j.out1 = uni; j.method = method;
    run_threads(&j, nthreads, pair_worker);
}

/* Per-polygon pixel area and MBR (mbr as int32 [4n]: min x, min y, max x, max y). */
void oracle_polygon_areas(const i64* off, const int32_t* xy, i64 n, i64* area, int32_t* mbr,
                          int method, int nthreads)
{
    job_t j;
    memset(&j, 0, sizeof j);
    j.off_a = off; j.xy_a = xy; j.n = n; j.out0 = area; j.out1 = (i64*)mbr; j.method = method;
    run_threads(&j, nthreads, area_worker);
}

/* Candidate pairs by brute force within each tile: every (a, b) with tile_a[a] == tile_b[b] whose
 * closed MBRs overlap (ax0 <= bx1, bx0 <= ax1, ay0 <= by1, by0 <= ay1), in ascending (a, b) order.
 * Writes at most cap pairs and returns the total count. Tile ids must be non-decreasing in both
 * sets (returns -1 otherwise). */
i64 oracle_candidate_pairs(const int32_t* mbr_a, const int32_t* tile_a, i64 na,
                           const int32_t* mbr_b, const int32_t* tile_b, i64 nb,
                           i64* pa, i64* pb, i64 cap)
{
    for (i64 i = 1; i < na; ++i) if (tile_a[i] < tile_a[i - 1]) return -1;
    for (i64 i = 1; i < nb; ++i) if (tile_b[i] < tile_b[i - 1]) return -1;
    i64 cnt = 0, b_lo = 0;
    for (i64 a = 0; a < na; ++a) {
        const int32_t t = tile_a[a];
        while (b_lo < nb && tile_b[b_lo] < t) ++b_lo;
        const int32_t* A = mbr_a + 4 * a;
        for (i64 b = b_lo; b < nb && tile_b[b] == t; ++b) {
            const int32_t* B = mbr_b + 4 * b;
            if (A[0] <= B[2] && B[0] <= A[2] && A[1] <= B[3] && B[1] <= A[3]) {
                if (cnt < cap) { pa[cnt] = a; pb[cnt] = b; }
                ++cnt;
            }
        }
    }
    return cnt;
}

/* ------------------------------------------------------------------------------------------- */
/* ST_Touches by the rule stated with the other operators of Sec. 3.4 ("Implications of PixelBox  */
/* to other spatial operators"): two polygons touch when no edge of one crosses an edge of the    */
/* other, no vertex of one lies within the other, and at least one vertex of one lies on an edge  */
/* of the other. Read exactly, with integer orientation tests (|coordinates| <= 2^28, products    */
/* below 2^62): "crosses" = the two segments' interiors cross at one point (each segment's        */
/* endpoints strictly on opposite sides of the other's line); "lies within" = strictly inside by  */
/* the even-odd rule and on no edge; "lies on an edge" = on the closed segment.                   */
/* ------------------------------------------------------------------------------------------- */
static int orient_sign(i64 ax, i64 ay, i64 bx, i64 by, i64 cx, i64 cy)
{
    const i64 v = (bx - ax) * (cy - ay) - (by - ay) * (cx - ax);
    return (v > 0) - (v < 0);
}

static int on_segment(i64 ax, i64 ay, i64 bx, i64 by, i64 px, i64 py)
{
    if (orient_sign(ax, ay, bx, by, px, py) != 0) return 0;
    return px >= (ax < bx ? ax : bx) && px <= (ax < bx ? bx : ax) && py >= (ay < by ? ay : by) &&
           py <= (ay < by ? by : ay);
}

/* 1 if (px, py) is on the boundary of the ring, else 0. */
static int on_boundary(const int32_t* xy, i64 nv, i64 px, i64 py)
{
    for (i64 e = 0; e < nv; ++e) {
        const i64 f = (e + 1 == nv) ? 0 : e + 1;
        if (on_segment(xy[2 * e], xy[2 * e + 1], xy[2 * f], xy[2 * f + 1], px, py)) return 1;
    }
    return 0;
}

/* Even-odd parity of a point not on the boundary: count edges whose half-open y-range
 * [min y, max y) contains py and whose x at height py is greater than px. */
static int point_inside(const int32_t* xy, i64 nv, i64 px, i64 py)
{
    int par = 0;
    for (i64 e = 0; e < nv; ++e) {
        const i64 f = (e + 1 == nv) ? 0 : e + 1;
        i64 ax = xy[2 * e], ay = xy[2 * e + 1], bx = xy[2 * f], by = xy[2 * f + 1];
        if (ay > by) { i64 t = ax; ax = bx; bx = t; t = ay; ay = by; by = t; }
        if (!(ay <= py && py < by)) continue;
        /* the edge's x at height py, ax + (py - ay)(bx - ax)/(by - ay), exceeds px; by > ay here */
        if ((px - ax) * (by - ay) < (py - ay) * (bx - ax)) par ^= 1;
    }
    return par;
}

int oracle_touches(const int32_t* xp, i64 np, const int32_t* xq, i64 nq)
{
    int vertex_on_edge = 0;
    for (i64 e = 0; e < np; ++e) {
        const i64 f = (e + 1 == np) ? 0 : e + 1;
        const i64 ax = xp[2 * e], ay = xp[2 * e + 1], bx = xp[2 * f], by = xp[2 * f + 1];
        for (i64 g = 0; g < nq; ++g) {
            const i64 h = (g + 1 == nq) ? 0 : g + 1;
            const i64 cx = xq[2 * g], cy = xq[2 * g + 1], dx = xq[2 * h], dy = xq[2 * h + 1];
            const int o1 = orient_sign(ax, ay, bx, by, cx, cy), o2 = orient_sign(ax, ay, bx, by, dx, dy);
            const int o3 = orient_sign(cx, cy, dx, dy, ax, ay), o4 = orient_sign(cx, cy, dx, dy, bx, by);
            if (o1 * o2 < 0 && o3 * o4 < 0) return 0;            /* edges cross */
        }
    }
    for (int side = 0; side < 2; ++side) {
        const int32_t* u = side ? xq : xp;
        const int32_t* w = side ? xp : xq;
        const i64 nu = side ? nq : np, nw = side ? np : nq;
        for (i64 k = 0; k < nu; ++k) {
            const i64 px = u[2 * k], py = u[2 * k + 1];
            if (on_boundary(w, nw, px, py)) { vertex_on_edge = 1; continue; }
            if (point_inside(w, nw, px, py)) return 0;           /* a vertex within the other */
        }
    }
    return vertex_on_edge;
}
