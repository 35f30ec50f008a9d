/*
 * afps_oracle.c -- plain, slow CPU oracle for FPS, AFPS and NPDU-AFPS.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package's smoke check
 * and the benchmark's CPU-baseline leg may load this library.  It shares no
 * code, header, table or constant with the CUDA path and must never be used
 * as a fallback for it.
 *
 * Build with contraction off (gcc -O2 -ffp-contract=off): every product and
 * sum below is rounded on its own, exactly like the CUDA path, so that the
 * int32 sample indices of the two can be compared bit for bit.
 *
 * What it computes (arXiv 2208.08795):
 *   - Algorithm 1 (plain FPS): keep a running distance array initialised to
 *     1e10; after each new sample, every point j takes
 *     Distance[j] = dist if dist <= Distance[j]; the next sample is the
 *     argmax of Distance.  The squared Euclidean distance is used: the
 *     argmax is the same as for the true distance in exact arithmetic, and
 *     the squared form (dx*dx + dy*dy) + dz*dz is what both sides round.
 *   - Sec. III-B (AFPS): the cloud is cut by storage position into M
 *     contiguous sectors and each sector runs its own FPS for C/M samples.
 *     M = 1 is plain FPS; M = C takes one sample per sector.
 *   - Sec. III-C (NPDU): after each new sample only the points stored next to
 *     it are updated, a window of constant size k, applied within each sector.
 *
 * Readings taken where the paper is silent (listed with the design notes):
 *   R1 sector s covers [floor(s*N/M), floor((s+1)*N/M)) and takes
 *      floor((s+1)*C/M) - floor(s*C/M) samples, written at output offset
 *      floor(s*C/M), in selection order (sector-major output);
 *   R2 the start index lies in sector s0 at offset r; every sector starts at
 *      its own offset min(r, n_s - 1);
 *   R3 the NPDU window is [p - floor(k/2), p + (k - floor(k/2))] clipped to
 *      the sector (k neighbours plus the sample itself); k = 0 means "no NPDU";
 *   R4 ties in the argmax go to the lowest index;
 *   R5 no first full pass under NPDU: points never inside a window keep 1e10.
 * Two other readings of Sec. III-C are available as method options:
 *   ORACLE_NPDU_FULL_FIRST_PASS   the first update (after the first sample)
 *                                 reaches the whole sector, later ones the
 *                                 window only;
 *   ORACLE_NPDU_WINDOW_HAS_SAMPLE k counts the sample itself: the window is
 *                                 [p - floor((k-1)/2), p + (k-1) - floor((k-1)/2)].
 */
#include <stdint.h>
#include <stdlib.h>
#include <math.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID_ARG (-1)
#define ORACLE_ERR_SECTOR_TOO_SMALL (-2)
#define ORACLE_ERR_NO_MEMORY (-3)

#define ORACLE_NPDU_FULL_FIRST_PASS 1u
#define ORACLE_NPDU_WINDOW_HAS_SAMPLE 2u

/* Algorithm 1, initial value of the Distance array. */
#define ORACLE_DIST_INIT_F32 1e10f
#define ORACLE_DIST_INIT_F64 1e10

/* Sector s of an AFPS run (Sec. III-B, reading R1). */
static void oracle_sector(int64_t N, int64_t C, int64_t M, int64_t s,
                          int64_t* lo, int64_t* n, int64_t* off, int64_t* c)
{
    int64_t lo0 = (s * N) / M;
    int64_t lo1 = ((s + 1) * N) / M;
    int64_t off0 = (s * C) / M;
    int64_t off1 = ((s + 1) * C) / M;
    *lo = lo0;
    *n = lo1 - lo0;
    *off = off0;
    *c = off1 - off0;
}

/* Argument checks shared by both precisions; returns ORACLE_OK or an error. */
static int oracle_check(int64_t N, int32_t C, int32_t M, int32_t k, int64_t start_idx)
{
    if (N < 1 || C < 1 || (int64_t)C > N || M < 1 || M > C || k < 0 ||
        start_idx < 0 || start_idx >= N)
        return ORACLE_ERR_INVALID_ARG;
    for (int64_t s = 0; s < M; ++s) {
        int64_t lo, n, off, c;
        oracle_sector(N, C, M, s, &lo, &n, &off, &c);
        if (c > n) return ORACLE_ERR_SECTOR_TOO_SMALL;
    }
    return ORACLE_OK;
}

/* Reading R2: the sector holding start_idx, and the offset inside it. */
static void oracle_start_offset(int64_t N, int64_t C, int64_t M, int64_t start_idx,
                                int64_t* r_out)
{
    for (int64_t s = 0; s < M; ++s) {
        int64_t lo, n, off, c;
        oracle_sector(N, C, M, s, &lo, &n, &off, &c);
        if (start_idx >= lo && start_idx < lo + n) {
            *r_out = start_idx - lo;
            return;
        }
    }
    *r_out = 0;
}

/*
 * Sector table for tests: lo[M+1], off[M+1], first[M] (global index of each
 * sector's first sample).  Returns ORACLE_OK or an error code.
 */
int oracle_sector_table(int64_t N, int32_t C, int32_t M, int64_t start_idx,
                        int64_t* lo, int64_t* off, int64_t* first)
{
    int rc = oracle_check(N, C, M, 0, start_idx);
    if (rc != ORACLE_OK) return rc;
    int64_t r;
    oracle_start_offset(N, C, M, start_idx, &r);
    for (int64_t s = 0; s < M; ++s) {
        int64_t l, n, o, c;
        oracle_sector(N, C, M, s, &l, &n, &o, &c);
        lo[s] = l;
        off[s] = o;
        first[s] = l + (r < n - 1 ? r : n - 1);
    }
    lo[M] = N;
    off[M] = C;
    return ORACLE_OK;
}

/*
 * One sector's FPS loop in fp32 (Algorithm 1 restricted to the sector, with
 * the NPDU window of Sec. III-C when k > 0).  P points at the sector's first
 * point (xyz interleaved), n points, c samples, first = local start index.
 * D is scratch of n floats.  Writes c global indices (lo + local) to out.
 */
static void oracle_sector_fps_f32(const float* P, int64_t lo, int64_t n, int64_t c,
                                  int64_t first, int32_t k, int64_t kl, int64_t kr,
                                  int full_first, float* D, int32_t* out)
{
    for (int64_t j = 0; j < n; ++j) D[j] = ORACLE_DIST_INIT_F32;
    int64_t p = first;
    for (int64_t t = 0; t < c; ++t) {
        out[t] = (int32_t)(lo + p);
        if (t == c - 1) break;
        /* points whose distance is updated this iteration */
        int64_t a = 0, b = n - 1;
        if (k > 0 && !(full_first && t == 0)) {
            a = p - kl;
            b = p + kr;
            if (a < 0) a = 0;
            if (b > n - 1) b = n - 1;
        }
        const float px = P[3 * p + 0];
        const float py = P[3 * p + 1];
        const float pz = P[3 * p + 2];
        for (int64_t j = a; j <= b; ++j) {
            float dx = P[3 * j + 0] - px;
            float dy = P[3 * j + 1] - py;
            float dz = P[3 * j + 2] - pz;
            float dist = (dx * dx + dy * dy) + dz * dz;
            if (dist <= D[j]) D[j] = dist;
        }
        /* next sample: argmax of Distance, lowest index on ties */
        int64_t best = 0;
        for (int64_t j = 1; j < n; ++j)
            if (D[j] > D[best]) best = j;
        p = best;
    }
}

/* The same loop in fp64, on inputs widened from fp32. */
static void oracle_sector_fps_f64(const float* P, int64_t lo, int64_t n, int64_t c,
                                  int64_t first, int32_t k, int64_t kl, int64_t kr,
                                  int full_first, double* D, int32_t* out)
{
    for (int64_t j = 0; j < n; ++j) D[j] = ORACLE_DIST_INIT_F64;
    int64_t p = first;
    for (int64_t t = 0; t < c; ++t) {
        out[t] = (int32_t)(lo + p);
        if (t == c - 1) break;
        int64_t a = 0, b = n - 1;
        if (k > 0 && !(full_first && t == 0)) {
            a = p - kl;
            b = p + kr;
            if (a < 0) a = 0;
            if (b > n - 1) b = n - 1;
        }
        const double px = (double)P[3 * p + 0];
        const double py = (double)P[3 * p + 1];
        const double pz = (double)P[3 * p + 2];
        for (int64_t j = a; j <= b; ++j) {
            double dx = (double)P[3 * j + 0] - px;
            double dy = (double)P[3 * j + 1] - py;
            double dz = (double)P[3 * j + 2] - pz;
            double dist = (dx * dx + dy * dy) + dz * dz;
            if (dist <= D[j]) D[j] = dist;
        }
        int64_t best = 0;
        for (int64_t j = 1; j < n; ++j)
            if (D[j] > D[best]) best = j;
        p = best;
    }
}

/* Window sides of the NPDU reading selected by `method`. */
static void oracle_window(int32_t k, uint32_t method, int64_t* kl, int64_t* kr)
{
    if (method & ORACLE_NPDU_WINDOW_HAS_SAMPLE) {
        *kl = (k - 1) / 2;
        *kr = (k - 1) - (k - 1) / 2;
    } else {
        *kl = k / 2;
        *kr = k - k / 2;
    }
}

/*
 * NPDU-AFPS on one cloud in fp32.  xyz: N points, xyz interleaved (host).
 * C samples, M sectors, k = NPDU window (0 = off), start_idx in [0, N).
 * out: C int32 global indices, sector-major.  Nothing is written on error.
 * M = 1, k = 0 is plain FPS (Algorithm 1 with a fixed start).
 */
int oracle_afps_ex_f32(const float* xyz, int64_t N, int32_t C, int32_t M, int32_t k,
                       int64_t start_idx, uint32_t method, int32_t* out)
{
    int rc = oracle_check(N, C, M, k, start_idx);
    if (rc != ORACLE_OK) return rc;
    if (!xyz || !out || method > 3u) return ORACLE_ERR_INVALID_ARG;
    int64_t r, kl, kr;
    oracle_start_offset(N, C, M, start_idx, &r);
    oracle_window(k, method, &kl, &kr);
    float* D = (float*)malloc(sizeof(float) * (size_t)N);
    if (!D) return ORACLE_ERR_NO_MEMORY;
    for (int64_t s = 0; s < M; ++s) {
        int64_t lo, n, off, c;
        oracle_sector(N, C, M, s, &lo, &n, &off, &c);
        int64_t first = r < n - 1 ? r : n - 1;
        oracle_sector_fps_f32(xyz + 3 * lo, lo, n, c, first, k, kl, kr,
                              (method & ORACLE_NPDU_FULL_FIRST_PASS) != 0, D, out + off);
    }
    free(D);
    return ORACLE_OK;
}

int oracle_afps_f32(const float* xyz, int64_t N, int32_t C, int32_t M, int32_t k,
                    int64_t start_idx, int32_t* out)
{
    return oracle_afps_ex_f32(xyz, N, C, M, k, start_idx, 0u, out);
}

/* The same method in fp64 (for agreement rates and coverage radii). */
int oracle_afps_ex_f64(const float* xyz, int64_t N, int32_t C, int32_t M, int32_t k,
                       int64_t start_idx, uint32_t method, int32_t* out)
{
    int rc = oracle_check(N, C, M, k, start_idx);
    if (rc != ORACLE_OK) return rc;
    if (!xyz || !out || method > 3u) return ORACLE_ERR_INVALID_ARG;
    int64_t r, kl, kr;
    oracle_start_offset(N, C, M, start_idx, &r);
    oracle_window(k, method, &kl, &kr);
    double* D = (double*)malloc(sizeof(double) * (size_t)N);
    if (!D) return ORACLE_ERR_NO_MEMORY;
    for (int64_t s = 0; s < M; ++s) {
        int64_t lo, n, off, c;
        oracle_sector(N, C, M, s, &lo, &n, &off, &c);
        int64_t first = r < n - 1 ? r : n - 1;
        oracle_sector_fps_f64(xyz + 3 * lo, lo, n, c, first, k, kl, kr,
                              (method & ORACLE_NPDU_FULL_FIRST_PASS) != 0, D, out + off);
    }
    free(D);
    return ORACLE_OK;
}

int oracle_afps_f64(const float* xyz, int64_t N, int32_t C, int32_t M, int32_t k,
                    int64_t start_idx, int32_t* out)
{
    return oracle_afps_ex_f64(xyz, N, C, M, k, start_idx, 0u, out);
}

/*
 * Coverage radius of a sample set, in fp64: max over all points j of the
 * Euclidean distance to the nearest sample.  This is the quantity FPS greedily
 * shrinks (property P1 of Sec. II-B); it scores a sample set without a
 * trained network.  Returns -1 on bad arguments.
 */
double oracle_coverage_radius(const float* xyz, int64_t N, const int32_t* idx, int32_t C)
{
    if (!xyz || !idx || N < 1 || C < 1) return -1.0;
    double worst = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        double best = INFINITY;
        for (int32_t s = 0; s < C; ++s) {
            int64_t q = idx[s];
            if (q < 0 || q >= N) return -1.0;
            double dx = (double)xyz[3 * j + 0] - (double)xyz[3 * q + 0];
            double dy = (double)xyz[3 * j + 1] - (double)xyz[3 * q + 1];
            double dz = (double)xyz[3 * j + 2] - (double)xyz[3 * q + 2];
            double d = (dx * dx + dy * dy) + dz * dz;
            if (d < best) best = d;
        }
        if (best > worst) worst = best;
    }
    return sqrt(worst);
}

/*
 * Ball query (the grouping step that follows sampling in a PointNet++ set
 * abstraction, Sec. I-II; the paper does not define it, this is the usual
 * reading): for each of the C centroids (indices into the cloud), the first
 * K points in storage order whose squared distance to the centroid,
 * (dx*dx + dy*dy) + dz*dz in fp32, is below radius*radius (fp32); when fewer
 * than K are found the remaining slots repeat the first one found (or -1 if
 * none).  out: C x K int32.  Returns ORACLE_OK or ORACLE_ERR_INVALID_ARG.
 */
int oracle_ball_query(const float* xyz, int64_t N, const int32_t* centroids, int32_t C,
                      float radius, int32_t K, int32_t* out)
{
    if (!xyz || !centroids || !out || N < 1 || C < 0 || K < 1 || !(radius > 0.0f))
        return ORACLE_ERR_INVALID_ARG;
    const float r2 = radius * radius;
    for (int32_t s = 0; s < C; ++s) {
        const int64_t q = centroids[s];
        if (q < 0 || q >= N) return ORACLE_ERR_INVALID_ARG;
        const float cx = xyz[3 * q + 0], cy = xyz[3 * q + 1], cz = xyz[3 * q + 2];
        int32_t cnt = 0;
        for (int64_t j = 0; j < N && cnt < K; ++j) {
            float dx = xyz[3 * j + 0] - cx;
            float dy = xyz[3 * j + 1] - cy;
            float dz = xyz[3 * j + 2] - cz;
            float d2 = (dx * dx + dy * dy) + dz * dz;
            if (d2 < r2) out[(int64_t)s * K + cnt++] = (int32_t)j;
        }
        const int32_t fill = cnt > 0 ? out[(int64_t)s * K] : -1;
        for (int32_t i = cnt; i < K; ++i) out[(int64_t)s * K + i] = fill;
    }
    return ORACLE_OK;
}

/*
 * k nearest neighbours (the other grouping step used after sampling in
 * point-cloud networks, Sec. I-II; the paper does not define it, this is the
 * plain reading): for each of the C centroids, the K points with the
 * smallest squared distance (dx*dx + dy*dy) + dz*dz in fp32, ties to the
 * lower index, listed nearest first.  Every point's key (distance, index)
 * is formed and the keys are sorted; the first K are kept.  out: C x K
 * int32; d2 (optional): the matching squared distances.  Needs 1 <= K <= N.
 * Returns ORACLE_OK, ORACLE_ERR_INVALID_ARG or ORACLE_ERR_NO_MEMORY.
 */
typedef struct {
    float d;
    int64_t j;
} oracle_knn_key;

static int oracle_knn_cmp(const void* a, const void* b)
{
    const oracle_knn_key* x = (const oracle_knn_key*)a;
    const oracle_knn_key* y = (const oracle_knn_key*)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->j > y->j) - (x->j < y->j);
}

int oracle_knn(const float* xyz, int64_t N, const int32_t* centroids, int32_t C, int32_t K,
               int32_t* out, float* d2)
{
    if (!xyz || !centroids || !out || N < 1 || C < 0 || K < 1 || K > N)
        return ORACLE_ERR_INVALID_ARG;
    oracle_knn_key* keys = (oracle_knn_key*)malloc((size_t)N * sizeof(oracle_knn_key));
    if (!keys) return ORACLE_ERR_NO_MEMORY;
    for (int32_t s = 0; s < C; ++s) {
        const int64_t q = centroids[s];
        if (q < 0 || q >= N) {
            free(keys);
            return ORACLE_ERR_INVALID_ARG;
        }
        const float cx = xyz[3 * q + 0], cy = xyz[3 * q + 1], cz = xyz[3 * q + 2];
        for (int64_t j = 0; j < N; ++j) {
            float ex = xyz[3 * j + 0] - cx;
            float ey = xyz[3 * j + 1] - cy;
            float ez = xyz[3 * j + 2] - cz;
            keys[j].d = (ex * ex + ey * ey) + ez * ez;
            keys[j].j = j;
        }
        qsort(keys, (size_t)N, sizeof(oracle_knn_key), oracle_knn_cmp);
        for (int32_t i = 0; i < K; ++i) {
            out[(int64_t)s * K + i] = (int32_t)keys[i].j;
            if (d2) d2[(int64_t)s * K + i] = keys[i].d;
        }
    }
    free(keys);
    return ORACLE_OK;
}
