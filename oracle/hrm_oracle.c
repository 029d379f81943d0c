/*
 * hrm_oracle.c -- brute-force CPU oracle for the exact running median.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only tests/, the smoke check and the bench's CPU-baseline
 * leg use it.  It shares no code, header, table or helper with the CUDA path.
 *
 * What it computes (Section II, definition of the median element of a set and
 * of the running/moving median): for every output point the window of
 * n = 2r+1 pixels per axis is centred on the point, coordinates outside the
 * image are clamped to the nearest edge (replicate border; clamped pixels are
 * counted with multiplicity, so every window holds exactly N = n^dims values),
 * and the output is the element of rank `rank` (0-based) of the window sorted
 * ascending.  The median is rank (N-1)/2, i.e. the "n^2/2 position" of the
 * sorted window (Section II, straight-forward implementation), which for odd N
 * is the unique middle element.  Section III (proof of get_order_statistic)
 * states that the hierarchical method returns exactly this K-th element of the
 * sorted list, and Section I / IV state that the filter's results equal any
 * other median filter's, so the oracle is the definition written out.
 *
 * Two interchangeable selection steps are provided:
 *   method 0: full sort of the window with the C library qsort
 *             (Section II, "sorting all values inside the window");
 *   method 1: Quickselect (Section II, Floyd's selection that places only the
 *             k-th smallest element), written plainly below.
 * The tests check that both give identical outputs.
 *
 * Parity status: pinned (hand-worked windows, closed forms, invariants,
 * threshold decomposition and scipy.ndimage on the CPU test suite).
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint32_t load_px(const unsigned char* base, int es)
{
    if (es == 1) return *base;
    uint16_t v;
    memcpy(&v, base, 2);
    return v;
}

static inline void store_px(unsigned char* base, int es, uint32_t v)
{
    if (es == 1) { *base = (unsigned char)v; return; }
    uint16_t w = (uint16_t)v;
    memcpy(base, &w, 2);
}

static inline long clampl(long v, long lo, long hi)
{
    return v < lo ? lo : (v > hi ? hi : v);
}

static int cmp_u32(const void* a, const void* b)
{
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* Quickselect with a middle pivot and two-sided partition: after each pass the
 * prefix [lo, j] holds values <= pivot, the suffix [i, hi] values >= pivot and
 * anything strictly between equals the pivot, so the k-th element lies in
 * whichever part contains index k. */
static uint32_t quickselect(uint32_t* a, long n, long k)
{
    long lo = 0, hi = n - 1;
    while (lo < hi) {
        uint32_t pivot = a[lo + (hi - lo) / 2];
        long i = lo, j = hi;
        while (i <= j) {
            while (a[i] < pivot) i++;
            while (a[j] > pivot) j--;
            if (i <= j) {
                uint32_t t = a[i];
                a[i] = a[j];
                a[j] = t;
                i++;
                j--;
            }
        }
        if (k <= j) hi = j;
        else if (k >= i) lo = i;
        else return a[k];
    }
    return a[k];
}

static uint32_t kth(uint32_t* buf, long n, long k, int method)
{
    if (method == 0) {
        qsort(buf, (size_t)n, sizeof(uint32_t), cmp_u32);
        return buf[k];
    }
    return quickselect(buf, n, k);
}

/* One output point of a (W,H,D) volume; D == 1 with rz == 0 is the 2D case. */
typedef struct {
    const unsigned char* src;
    size_t pitch, slice;
    int es, W, H, D, r, rz;
} vol_t;

static uint32_t point_value(const vol_t* v, long x, long y, long z, long rank,
                            int method, uint32_t* buf)
{
    long cnt = 0;
    for (long dz = -v->rz; dz <= v->rz; ++dz) {
        long zz = clampl(z + dz, 0, v->D - 1);
        for (long dy = -v->r; dy <= v->r; ++dy) {
            long yy = clampl(y + dy, 0, v->H - 1);
            const unsigned char* row = v->src + (size_t)zz * v->slice + (size_t)yy * v->pitch;
            for (long dx = -v->r; dx <= v->r; ++dx) {
                long xx = clampl(x + dx, 0, v->W - 1);
                buf[cnt++] = load_px(row + (size_t)xx * v->es, v->es);
            }
        }
    }
    return kth(buf, cnt, rank, method);
}

static long window_count(int r, int rz)
{
    long n = 2L * r + 1, nz = 2L * rz + 1;
    return n * n * nz;
}

/* ---- threaded drivers ------------------------------------------------- */

typedef struct {
    const vol_t* v;
    unsigned char* dst;
    size_t dpitch, dslice;
    long rank;
    int method;
    long first, last; /* range of (z*H + y) rows, or of point indices */
    const int *xs, *ys, *zs;
    uint32_t* out;
    int err;
} job_t;

static void* run_rows(void* p)
{
    job_t* j = (job_t*)p;
    const vol_t* v = j->v;
    uint32_t* buf = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)window_count(v->r, v->rz));
    if (!buf) { j->err = 1; return NULL; }
    for (long zy = j->first; zy < j->last; ++zy) {
        long z = zy / v->H, y = zy % v->H;
        unsigned char* drow = j->dst + (size_t)z * j->dslice + (size_t)y * j->dpitch;
        for (long x = 0; x < v->W; ++x)
            store_px(drow + (size_t)x * v->es, v->es,
                     point_value(v, x, y, z, j->rank, j->method, buf));
    }
    free(buf);
    return NULL;
}

static void* run_points(void* p)
{
    job_t* j = (job_t*)p;
    const vol_t* v = j->v;
    uint32_t* buf = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)window_count(v->r, v->rz));
    if (!buf) { j->err = 1; return NULL; }
    for (long i = j->first; i < j->last; ++i)
        j->out[i] = point_value(v, j->xs[i], j->ys[i], j->zs ? j->zs[i] : 0, j->rank, j->method, buf);
    free(buf);
    return NULL;
}

static int spawn(job_t* jobs, int nthreads, long total, void* (*fn)(void*))
{
    pthread_t th[256];
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    if (nthreads > total) nthreads = (int)(total > 0 ? total : 1);
    long per = (total + nthreads - 1) / nthreads;
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        jobs[t] = jobs[0];
        jobs[t].first = t * per < total ? t * per : total;
        jobs[t].last = (t + 1) * per < total ? (t + 1) * per : total;
        jobs[t].err = 0;
    }
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, fn, &jobs[t]) != 0) break;
        started++;
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    if (started != nthreads) return -2;
    for (int t = 0; t < nthreads; ++t)
        if (jobs[t].err) return -2;
    return 0;
}

static int check_args(int es, int W, int H, int D, int r, long rank, int rz)
{
    if (es != 1 && es != 2) return -1;
    if (W < 1 || H < 1 || D < 1 || r < 0 || rz < 0) return -1;
    long N = window_count(r, rz);
    if (rank < -1 || rank >= N) return -1;
    return 0;
}

/* 2D filter of a whole image.  Pitches are in bytes.  rank < 0 selects the
 * median (N-1)/2.  Returns 0, -1 on bad arguments, -2 on allocation failure. */
int oracle_filter2d(int es, const void* src, size_t src_pitch, void* dst, size_t dst_pitch,
                    int W, int H, int r, long rank, int method, int nthreads)
{
    if (check_args(es, W, H, 1, r, rank, 0)) return -1;
    if (rank < 0) rank = (window_count(r, 0) - 1) / 2;
    vol_t v = {(const unsigned char*)src, src_pitch, 0, es, W, H, 1, r, 0};
    job_t jobs[256];
    memset(jobs, 0, sizeof(jobs));
    jobs[0].v = &v;
    jobs[0].dst = (unsigned char*)dst;
    jobs[0].dpitch = dst_pitch;
    jobs[0].rank = rank;
    jobs[0].method = method;
    return spawn(jobs, nthreads, (long)H, run_rows);
}

/* 3D filter with a cubic window (radius r along x, y and z). */
int oracle_filter3d(int es, const void* src, size_t src_pitch, size_t src_slice,
                    void* dst, size_t dst_pitch, size_t dst_slice,
                    int W, int H, int D, int r, long rank, int method, int nthreads)
{
    if (check_args(es, W, H, D, r, rank, r)) return -1;
    if (rank < 0) rank = (window_count(r, r) - 1) / 2;
    vol_t v = {(const unsigned char*)src, src_pitch, src_slice, es, W, H, D, r, r};
    job_t jobs[256];
    memset(jobs, 0, sizeof(jobs));
    jobs[0].v = &v;
    jobs[0].dst = (unsigned char*)dst;
    jobs[0].dpitch = dst_pitch;
    jobs[0].dslice = dst_slice;
    jobs[0].rank = rank;
    jobs[0].method = method;
    return spawn(jobs, nthreads, (long)H * D, run_rows);
}

/* Selected output points only (for full-size workloads): out[i] is the
 * filter output at (xs[i], ys[i], zs[i]); zs may be NULL for 2D (depth 1,
 * rz = 0).  For 3D pass D > 1 or rz = r. */
int oracle_points(int es, const void* src, size_t src_pitch, size_t src_slice,
                  int W, int H, int D, int r, int rz, long rank,
                  const int* xs, const int* ys, const int* zs, long npts,
                  uint32_t* out, int method, int nthreads)
{
    if (check_args(es, W, H, D, r, rank, rz)) return -1;
    if (rank < 0) rank = (window_count(r, rz) - 1) / 2;
    for (long i = 0; i < npts; ++i) {
        if (xs[i] < 0 || xs[i] >= W || ys[i] < 0 || ys[i] >= H) return -1;
        if (zs && (zs[i] < 0 || zs[i] >= D)) return -1;
    }
    if (npts == 0) return 0;
    vol_t v = {(const unsigned char*)src, src_pitch, src_slice, es, W, H, D, r, rz};
    job_t jobs[256];
    memset(jobs, 0, sizeof(jobs));
    jobs[0].v = &v;
    jobs[0].rank = rank;
    jobs[0].method = method;
    jobs[0].xs = xs;
    jobs[0].ys = ys;
    jobs[0].zs = zs;
    jobs[0].out = out;
    return spawn(jobs, nthreads, npts, run_points);
}
