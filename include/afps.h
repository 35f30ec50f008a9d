/*
 * afps.h -- C ABI of the GB300 (sm_103a) NPDU-AFPS library, libafps.so.
 *
 * The method (arXiv 2208.08795):
 *   - Farthest Point Sampling, Algorithm 1 (Sec. II-B): starting from one
 *     sample, keep each point's distance to the nearest sample so far
 *     (initially 1e10) and repeatedly take the farthest point;
 *   - AFPS, Sec. III-B: cut the cloud by storage position into M contiguous
 *     sectors and run FPS in each sector for C/M samples;
 *   - NPDU, Sec. III-C and Fig. 3: after each new sample update only the k
 *     points stored next to it, inside its own sector.
 *
 * Definitions fixed by this library where the paper leaves a choice:
 *   - distance: squared Euclidean distance in fp32, (dx*dx + dy*dy) + dz*dz,
 *     every product and sum rounded on its own (no fused multiply-add);
 *   - sector s of a cloud of N points with C samples and M sectors covers
 *     points [floor(s*N/M), floor((s+1)*N/M)) and takes
 *     c_s = floor((s+1)*C/M) - floor(s*C/M) samples, written to output slots
 *     [floor(s*C/M), floor((s+1)*C/M)) in the order they are selected;
 *   - start: start_idx lies in sector s0 at offset r; every sector starts at
 *     its own offset min(r, n_s - 1);
 *   - NPDU window of a sample at sector offset p: offsets
 *     [p - floor(k/2), p + k - floor(k/2)] clipped to the sector, i.e. k
 *     neighbours plus the sample itself; k = 0 disables NPDU;
 *   - no first full pass under NPDU: points never inside a window keep 1e10;
 *   - ties in the argmax go to the lowest index.
 * With M = 1 and k = 0 the result is plain FPS (Algorithm 1, fixed start).
 *
 * Conventions for every call:
 *   - xyz is an array of points, 3 consecutive float32 per point (x, y, z),
 *     4-byte aligned; coordinates must be finite.
 *   - Output indices are int32, relative to the first point of their cloud,
 *     sector-major (see above).
 *   - "d_" pointers are device memory of the context's device, "h_" pointers
 *     host memory.  The caller owns every buffer it passes; the context owns
 *     its workspace, graphs and tuning cache.
 *   - stream is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls are asynchronous on that stream unless stated.
 *   - Return value: AFPS_OK (0) or a negative AFPS_ERR_* code; the message of
 *     the last error is afps_last_error(ctx).  Nothing is written to any
 *     output on a validation error.
 *   - A context may be used from one host thread at a time, with any number
 *     of streams.  A call that uses the context's device workspace (the item
 *     table of a ragged batch, the work-queue counters of a batch larger than
 *     one wave of the grid) waits on the device for the previous call that
 *     used it, whatever its stream; other calls on different streams may run
 *     at the same time, which is how independent batches overlap.
 */
#ifndef AFPS_H
#define AFPS_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define AFPS_OK 0
#define AFPS_ERR_INVALID_ARG (-1)      /* bad pointer, size or parameter */
#define AFPS_ERR_SECTOR_TOO_SMALL (-2) /* some sector has c_s > n_s */
#define AFPS_ERR_NO_MEMORY (-3)        /* device or host allocation failed */
#define AFPS_ERR_TIMEOUT (-4)          /* a device-side wait ran out of time */
#define AFPS_ERR_CUDA (-5)             /* a CUDA runtime call failed */
#define AFPS_ERR_UNSUPPORTED (-6)      /* sector larger than AFPS_MAX_SECTOR_POINTS */

/* Largest sector (points) any kernel handles: 16 CTAs x 1024 threads x 8. */
#define AFPS_MAX_SECTOR_POINTS 131072

/* afps_config.flags */
#define AFPS_FLAG_GRAPH 1u     /* replay afps_sample_batched from cached CUDA graphs */
/* The first batched call with an argument set that has a shape class
 * without a tuned variant runs afps_autotune_batched on it (synchronously),
 * then samples as usual. */
#define AFPS_FLAG_AUTOTUNE 2u
/* Fault injection for tests of failure detection: the stage-in arms its
 * shared-memory barrier but never issues the bulk copy, so the bounded wait
 * runs out (after timeout_ns) and afps_sync returns AFPS_ERR_TIMEOUT.
 * Outputs of such calls are meaningless; the context stays usable.
 * After any timeout every kernel leaves its remaining work items undone
 * (nothing is computed on shared memory a copy may not have filled), and so
 * do later launches on the context until afps_sync has reported and
 * cleared the timeout: a stalled call costs a few timeouts, not one per
 * item or iteration. */
#define AFPS_FLAG_TEST_STALL_COPY 0x100u
/* Fault injection for tests of failure detection: in thread-block-cluster
 * kernels (plain FPS on large clouds) the last CTA of each cluster never
 * sends its records of the per-iteration argmax exchange, so the exchange's
 * bounded waits run out (after timeout_ns) and afps_sync returns
 * AFPS_ERR_TIMEOUT.  Outputs of such calls are meaningless; the context
 * stays usable. */
#define AFPS_FLAG_TEST_STALL_EXCHANGE 0x400u
/* Fault injection for tests of failure detection: every growth of the
 * context's device workspace (item tables, work-queue counters, staging and
 * scratch buffers) fails as it would on an exhausted device, so a call that
 * needs more workspace than the context already holds returns
 * AFPS_ERR_NO_MEMORY before it launches anything (its outputs untouched) and
 * the context stays usable.  (A failed device allocation returns
 * AFPS_ERR_NO_MEMORY with or without this flag.) */
#define AFPS_FLAG_TEST_FAIL_ALLOC 0x200u

typedef struct afps_ctx afps_ctx;

typedef struct afps_config {
    int32_t device;         /* CUDA device ordinal */
    uint32_t flags;         /* AFPS_FLAG_* */
    int64_t timeout_ns;     /* bound on each device-side wait; <= 0: 2 s */
    const char* tune_cache; /* autotuner cache file (read at create, written
                               by afps_save_tuning with a "# device" line
                               naming the GPU; a file from another kind of
                               GPU is ignored), or NULL */
} afps_config;

/*
 * Create a context on cfg->device (cfg may be NULL: device 0, no flags).
 * Allocates a small device status word and host staging.  On success *out
 * owns the context; free it with afps_destroy.
 */
int afps_create(afps_ctx** out, const afps_config* cfg);

/* Synchronise the context's device work and free everything it owns. */
void afps_destroy(afps_ctx* ctx);

/*
 * NPDU-AFPS of one cloud (Algorithm 1 + Sec. III-B + Sec. III-C).
 *   d_xyz        N points (device, read only)
 *   N            points, 1 <= N <= 2^31 - 1
 *   C            samples, 1 <= C <= N
 *   M            sectors, 1 <= M <= C; every sector needs c_s <= n_s
 *   npdu_window  k >= 0 (0 = no NPDU)
 *   start_idx    0 <= start_idx < N (Algorithm 1 draws it at random; the
 *                caller passes it)
 *   d_out        C int32 (device, written)
 * Sectors above AFPS_MAX_SECTOR_POINTS return AFPS_ERR_UNSUPPORTED.
 */
int afps_sample(afps_ctx* ctx, const float* d_xyz, int64_t N, int32_t C, int32_t M,
                int32_t npdu_window, int64_t start_idx, int32_t* d_out, void* stream);

/*
 * Readings of the NPDU window (Sec. III-C says only that the k points stored
 * next to each new sample are updated), for the _ex calls.  Method 0 is the
 * default reading above.  Bits:
 *   AFPS_METHOD_FULL_FIRST_PASS   the update after a sector's first sample
 *                                 reaches the whole sector; later updates the
 *                                 window only (no stride phase of untouched
 *                                 points);
 *   AFPS_METHOD_WINDOW_HAS_SAMPLE k counts the sample itself: the window is
 *                                 [p - floor((k-1)/2), p + (k-1) - floor((k-1)/2)].
 * Both apply only with k > 0.
 */
#define AFPS_METHOD_FULL_FIRST_PASS 1u
#define AFPS_METHOD_WINDOW_HAS_SAMPLE 2u
#define AFPS_METHOD_ALL 3u

/* afps_sample with an NPDU reading (AFPS_METHOD_* bits; 0 = afps_sample). */
int afps_sample_ex(afps_ctx* ctx, const float* d_xyz, int64_t N, int32_t C, int32_t M,
                   int32_t npdu_window, int64_t start_idx, uint32_t method, int32_t* d_out,
                   void* stream);

/*
 * A ragged batch of B clouds in one call, each cloud sampled exactly as
 * afps_sample would (Algorithm 1 in every sector, Sec. III-B; the NPDU
 * window of Sec. III-C).  The sectors of every cloud are independent (Sec.
 * III-B: each runs its own FPS loop), so all (cloud, sector) pairs of the
 * batch become work items of one kernel launch per kernel shape class
 * (sectors of similar size; NPDU classes that the window kernel serves share
 * one launch), distributed over the GPU by a work queue when there are more
 * items than resident warps.  Cloud b is points [h_pt_off[b], h_pt_off[b+1])
 * of d_xyz and writes h_C[b] indices at d_out[h_out_off[b]], relative to its
 * own first point.  Each cloud has its own C, M, k and start (h_* arrays of
 * B entries; h_pt_off and h_out_off of B+1 nondecreasing entries with
 * h_out_off[b+1] - h_out_off[b] >= h_C[b]).  With AFPS_FLAG_GRAPH the
 * launches are captured once per distinct argument set (pointers included)
 * and replayed; a context keeps up to 512 such graphs, evicting the least
 * recently used.  Host arrays are read before return.
 */
int afps_sample_batched(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off,
                        int32_t B, const int32_t* h_C, const int32_t* h_M,
                        const int32_t* h_win, const int64_t* h_start,
                        const int64_t* h_out_off, int32_t* d_out, void* stream);

/* afps_sample_batched with a per-cloud NPDU reading (h_method: B entries of
 * AFPS_METHOD_* bits). */
int afps_sample_batched_ex(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off,
                           int32_t B, const int32_t* h_C, const int32_t* h_M,
                           const int32_t* h_win, const int64_t* h_start,
                           const uint32_t* h_method, const int64_t* h_out_off, int32_t* d_out,
                           void* stream);

/*
 * afps_sample_batched on HOST buffers (h_pt_off[0] = h_out_off[0] = 0):
 * samples the h_pt_off[B] points of h_xyz, writes the h_out_off[B] indices to
 * h_out and waits for the stream before returning.  Pageable memory: copies
 * through context-owned device memory.  Page-locked memory with
 * AFPS_FLAG_GRAPH: one cached CUDA graph per argument set (pointers
 * included); when the buffers are mapped into the device's address space the
 * kernels read the points and write the indices in host memory directly (on
 * Grace-Blackwell over the coherent C2C link), otherwise the graph holds the
 * two copies around device staging.  Synchronous.
 */
int afps_sample_batched_host(afps_ctx* ctx, const float* h_xyz, const int64_t* h_pt_off,
                             int32_t B, const int32_t* h_C, const int32_t* h_M,
                             const int32_t* h_win, const int64_t* h_start,
                             const int64_t* h_out_off, int32_t* h_out, void* stream);

/*
 * afps_sample_batched_host without the final wait: the call returns once the
 * work is queued on the stream, so consecutive calls (on other buffers)
 * overlap.  Both buffers must be page-locked (AFPS_ERR_INVALID_ARG
 * otherwise) and stay untouched until the stream has reached the call
 * (afps_sync or a stream synchronisation); h_out holds the indices then.
 */
int afps_sample_batched_host_async(afps_ctx* ctx, const float* h_xyz, const int64_t* h_pt_off,
                                   int32_t B, const int32_t* h_C, const int32_t* h_M,
                                   const int32_t* h_win, const int64_t* h_start,
                                   const int64_t* h_out_off, int32_t* h_out, void* stream);

/*
 * Gather for chained sampling levels (the PointNet++ set-abstraction
 * hierarchy the paper targets, Sec. I-II): for each of B clouds, take the
 * samples d_sel[h_sel_off[b] .. h_sel_off[b+1]) (indices relative to the
 * cloud), sort them by ascending index (which keeps the storage order, and
 * hence the dimensional locality of Sec. III-A, for the next level) and write
 *   d_out_xyz   the sampled points in that order (3 floats each),
 *   d_out_frame d_in_frame[...] of those points in that order (the original
 *               frame index; d_in_frame NULL means the identity),
 *   d_sel_frame d_in_frame[sel] in the samples' own order (may be NULL).
 * Outputs use the h_sel_off layout and must not overlap the inputs.  Clouds
 * up to 65536 points.
 */
int afps_gather_levels(afps_ctx* ctx, int32_t B, const int64_t* h_in_pt_off,
                       const float* d_in_xyz, const int32_t* d_in_frame,
                       const int64_t* h_sel_off, const int32_t* d_sel,
                       float* d_out_xyz, int32_t* d_out_frame, int32_t* d_sel_frame,
                       void* stream);

/*
 * Sort keys for afps_sort_by_key.  AFPS_KEY_AZIMUTH is the "diamond angle"
 * of (x, y): a monotone stand-in for atan2(y, x) on [0, 4) defined, per
 * quadrant, as y/(x+y), 1 - x/(-x+y), 2 - y/(-x-y), 3 + x/(x-y) (each
 * operation rounded on its own; the origin maps to 0), so that it can be
 * reproduced exactly on any IEEE host.
 */
#define AFPS_KEY_X 0
#define AFPS_KEY_Y 1
#define AFPS_KEY_Z 2
#define AFPS_KEY_AZIMUTH 3

/*
 * Stable ascending sort of each cloud's points by a key, for input without
 * dimensional locality (Sec. III-A: AFPS and NPDU assume points stored next
 * to each other are close; binning or sorting restores that).  Cloud b is
 * points [h_pt_off[b], h_pt_off[b+1]) of d_xyz; its sorted points go to the
 * same range of d_xyz_sorted (must not overlap d_xyz) and d_perm[i] is the
 * cloud-relative index of the point now at position i.  Equal keys keep
 * their storage order; -0 and +0 are equal.  The context keeps 16 bytes of
 * device scratch per point.
 */
int afps_sort_by_key(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                     int32_t key, float* d_xyz_sorted, int32_t* d_perm, void* stream);

/*
 * Coverage radius of sample sets: for each of B clouds, d_radius[b] =
 * max over the cloud's points of the Euclidean distance to the nearest of
 * its samples d_sel[h_sel_off[b] .. h_sel_off[b+1]) (indices relative to the
 * cloud; out-of-range entries are clamped into it).  This is the quantity
 * FPS greedily shrinks (property P1, Sec. II-B) and scores sampling variants
 * without a trained network.  Computed in fp64 from the fp32 points with
 * separately rounded operations, so any IEEE host reproduces it exactly.
 * 1 <= B <= 65535.
 */
int afps_coverage_radius(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                         const int64_t* h_sel_off, const int32_t* d_sel, double* d_radius,
                         void* stream);

/*
 * Ball query, the grouping step that follows sampling in a PointNet++ set
 * abstraction (Sec. I-II; the paper does not define it, this is the usual
 * reading).  For each centroid d_sel[i] (cloud-relative, i in
 * [h_sel_off[b], h_sel_off[b+1]) for cloud b, clamped into the cloud):
 * d_group[i*K .. i*K+K) = the first K points of the cloud in storage order
 * whose fp32 squared distance (dx*dx + dy*dy) + dz*dz is below
 * radius*radius, the remaining slots repeating the first one found (-1 if
 * none).  sorted_axis = 0, 1, 2 promises the cloud is sorted ascending along
 * x, y or z, which lets the scan cover only the index range that can hold
 * hits (same result as a full scan); -1 scans every point.  1 <= B <= 65535.
 */
int afps_ball_query(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                    const int64_t* h_sel_off, const int32_t* d_sel, float radius, int32_t K,
                    int32_t sorted_axis, int32_t* d_group, void* stream);

/*
 * k nearest neighbours, the other grouping step used after sampling in
 * point-cloud networks (Sec. I-II; the paper does not define it, this is the
 * plain reading).  For each centroid d_sel[i] (cloud-relative, i in
 * [h_sel_off[b], h_sel_off[b+1]) for cloud b, clamped into the cloud):
 * d_group[i*K .. i*K+K) = the K points of the cloud with the smallest fp32
 * squared distance (dx*dx + dy*dy) + dz*dz (dx = point - centroid, every
 * operation rounded on its own), ties to the lower index, nearest first,
 * as cloud-relative indices; d_dist2 (may be NULL) receives the matching
 * squared distances.  sorted_axis = 0, 1, 2 promises the cloud is sorted
 * ascending along x, y or z, which lets the scan stop early on each side
 * (same result as a full scan); -1 scans every point.  Needs 1 <= K <= 64,
 * K <= every cloud's point count and 1 <= B <= 65535; device buffers are the
 * caller's; AFPS_ERR_INVALID_ARG otherwise (nothing launched).
 */
int afps_knn(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
             const int64_t* h_sel_off, const int32_t* d_sel, int32_t K, int32_t sorted_axis,
             int32_t* d_group, float* d_dist2, void* stream);

/*
 * Wait for the stream and report device-side errors recorded since the last
 * call (AFPS_ERR_TIMEOUT when a bounded wait gave up); clears them.
 */
int afps_sync(afps_ctx* ctx, void* stream);

/* Message of the last error on this context (never NULL; "" if none). */
const char* afps_last_error(const afps_ctx* ctx);

/*
 * Autotuner: time every kernel variant valid for the batch (same arguments
 * as afps_sample_batched; d_out is written with the correct result) and
 * remember the fastest per shape class.  Returns the number of classes
 * tuned, or a negative error.
 */
int afps_autotune_batched(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off,
                          int32_t B, const int32_t* h_C, const int32_t* h_M,
                          const int32_t* h_win, const int64_t* h_start,
                          const int64_t* h_out_off, int32_t* d_out, void* stream);

/* Write the tuning cache to path (NULL: the path given at create). */
int afps_save_tuning(afps_ctx* ctx, const char* path);

/*
 * Describe the kernel variant the planner would use for n_items sectors of
 * at most n_sector points and c_sector samples (for afps_sample, n_items is
 * M): writes a short text (kind, points per thread, warps per CTA, cluster
 * size) into buf.  Kinds: "warp" (a warp per sector, P points a lane),
 * "cta" / "cluster" (a CTA or a thread-block cluster of CS CTAs per sector),
 * "win" (NPDU window kernel, P rows of 32 points per warp buffer; "lean":
 * the round form with the fewest instructions) and "pair" (two NPDU
 * sectors per warp, P rows of 16 points per half).  "skip" marks row skips
 * outside the NPDU window.  Returns the text length or a negative error.
 */
int afps_describe_plan(afps_ctx* ctx, int64_t n_sector, int32_t c_sector,
                       int32_t npdu_window, int32_t n_items, char* buf, int32_t buf_len);

/*
 * Describe how afps_sample_batched would run an argument set (the same host
 * arrays) on this context: one entry per kernel launch, "<variant>
 * items=<n>", entries separated by "; " (e.g. "win P=9 W=8 items=17576").
 * Validates like afps_sample_batched; no device work.  Writes a
 * NUL-terminated text of at most buf_len bytes into buf and returns the
 * full text length, or a negative AFPS_ERR_* code.
 */
int afps_describe_batched(afps_ctx* ctx, const int64_t* h_pt_off, int32_t B,
                          const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
                          const int64_t* h_start, const int64_t* h_out_off, char* buf,
                          int32_t buf_len);

/* Number of kernel launches issued by this context since creation. */
int64_t afps_launch_count(const afps_ctx* ctx);

/*
 * afps_sample_batched for callers that cannot allocate.  The paper has no
 * counterpart: this is a deployment variant of the batched call above.
 *
 * Who needs it: code that may not call cudaMalloc (a plugin inside a host
 * framework that owns all device memory, a process under a fixed memory
 * budget or pool, a real-time loop that must not take allocator locks or
 * cause the implicit synchronisation an allocation can bring).  It takes no
 * context and allocates no device memory.  On the host heap it allocates
 * only on the first launch of each kernel variant on a device, where the
 * library records the kernel attributes it has set; a warm-up call with the
 * same shapes covers that.
 *
 * Arguments, layouts and results are those of afps_sample_batched; the
 * caller passes the input points and the output buffer.  The work-item table
 * (48 bytes per sector) lives in a static device array of
 * AFPS_NOALLOC_MAX_ITEMS items plus a 256-byte header (393,472 bytes, about
 * 384 KB) that every GPU loading the library holds until the process exits.
 * A batch with more sectors than that returns AFPS_ERR_SCRATCH_TOO_SMALL and
 * launches nothing.
 *
 * It runs on the current device.  The first call on a device looks up the
 * array's device address there (cudaGetSymbolAddress).  The table goes up
 * by cudaMemcpyAsync from the library's static host copy, which is pageable
 * memory, so a call may wait until the stream has reached it: it suits a
 * loop that must not allocate, not one that must never wait.  It must not
 * be captured into a CUDA graph (the copy would be recorded reading the host
 * copy at every replay, after later calls have overwritten it): on a stream
 * that is capturing it returns AFPS_ERR_INVALID_ARG and does nothing.  All
 * calls share the one array and it keeps the last call's table: calls whose
 * work overlaps on the GPU (different streams without ordering, or several
 * host threads) race on it.  Calls on one stream are ordered and safe.
 * Device-side wait timeouts are recorded in the array's status word, which
 * nothing reads back; use afps_sample_batched with afps_sync where such
 * reports matter.
 */
#define AFPS_NOALLOC_MAX_ITEMS 8192
#define AFPS_ERR_SCRATCH_TOO_SMALL (-7) /* batch exceeds AFPS_NOALLOC_MAX_ITEMS sectors */
int afps_sample_batched_noalloc(const float* d_xyz, const int64_t* h_pt_off, int32_t B,
                                const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
                                const int64_t* h_start, const int64_t* h_out_off,
                                int32_t* d_out, void* stream);

/* ----------------------------------------------------------------------------
 * Serving runtime: continuous batching of chained sampling requests.
 *
 * A request is one sensor frame (N points) and a chain of sampling levels,
 * the PointNet++ set-abstraction hierarchy the paper accelerates (Sec. I-II):
 * level 0 samples levels[0] points from the frame with NPDU-AFPS (M sectors,
 * window k), level l+1 samples levels[l+1] points from level l's samples
 * taken in ascending frame index (storage order kept, Sec. III-A).  The
 * result lists, per level, the frame indices of that level's samples in
 * emission (sector-major) order.
 *
 * Each afps_server_step admits queued requests while the device arena (the
 * HBM budget) and the slot count allow, then, levels_per_step times (default:
 * as many as there are levels), launches one batched sampling call over the
 * current level of every admitted request and one gather that builds every
 * next-level cloud on the device, and copies finished results to the host.
 * Requests at different levels share each launch; a request admitted while
 * others are on the GPU joins the next step.  Frames
 * and level clouds stay resident in the arena until their request finishes.
 * The host runs at most max_steps_ahead steps ahead of the GPU.
 * -------------------------------------------------------------------------- */
#define AFPS_SERVER_MAX_LEVELS 8
#define AFPS_ERR_BUSY (-8) /* afps_server_submit: the host queue is full */
/* afps_sync: a device-side index check failed (libraries built with
 * AFPS_DEBUG_CHECKS only: every sampling kernel checks its sector sizes and
 * indices, records a failure in the status word and clamps the index, so no
 * access leaves its buffer; the regular build compiles the checks out). */
#define AFPS_ERR_DEVICE_CHECK (-9)

typedef struct afps_server afps_server;

typedef struct afps_server_config {
    int64_t hbm_budget_bytes;  /* device arena for admitted requests (bytes) */
    int64_t max_queued;        /* frames waiting for admission; <= 0: 4096 */
    int32_t max_inflight;      /* admitted requests at once; <= 0: 256 */
    int32_t n_levels;          /* 1 .. AFPS_SERVER_MAX_LEVELS */
    int32_t levels[AFPS_SERVER_MAX_LEVELS]; /* samples per level */
    int32_t M;                 /* sectors per level (capped at the level's size) */
    int32_t npdu_window;       /* k >= 0 (0 = no NPDU) */
    int32_t max_steps_ahead;   /* <= 0: 2 */
    int32_t levels_per_step;   /* levels a step advances each admitted request by;
                                  <= 0: all (a request admitted by a step completes in it) */
    int64_t host_pool_bytes;   /* page-locked staging for queued frames; <= 0: 64 MiB */
} afps_server_config;

typedef struct afps_server_result {
    uint64_t tag;              /* the caller's tag from afps_server_submit */
    int32_t status;            /* AFPS_OK or an error code */
    int32_t n_levels;
    int32_t count[AFPS_SERVER_MAX_LEVELS];
    const int32_t* indices;    /* sum(count) frame indices, level after level; owned by
                                  the server, valid until the next afps_server_poll */
    double submit_ms, admit_ms, done_ms; /* server clock (afps_server_clock_ms) */
} afps_server_result;

/* Create a server on ctx's device, issuing its work on `stream` (NULL: a
 * stream of its own).  Allocates the arena and pinned result buffers.  When
 * every step runs all levels (levels_per_step <= 0 or >= n_levels),
 * consecutive steps share no request and the server alternates them between
 * `stream` (with ctx) and a second stream with a second context of its own
 * (ctx's flags, timeout and tuned variants; device errors still reach ctx's
 * status word, read by afps_sync on ctx), so that one step's frame copies
 * overlap the previous step's sampling; otherwise it uses `stream` alone.
 * ctx must outlive the server. */
int afps_server_create(afps_server** out, afps_ctx* ctx, const afps_server_config* cfg,
                       void* stream);

/* Queue one frame (N points, host memory, copied into the server's
 * page-locked pool before return, so that admission is an asynchronous DMA).
 * Needs levels[0] <= N <= 65536 and the request to fit the arena on its own.
 * Returns AFPS_ERR_BUSY when max_queued frames are waiting or the pool is
 * full. */
int afps_server_submit(afps_server* srv, const float* h_xyz, int64_t N, uint64_t tag);

/* Queue one frame that already lies in page-locked host memory, without
 * copying it: admission reads it there by DMA.  The frame must stay
 * allocated and unchanged until its result has been returned by
 * afps_server_poll.  Same limits as afps_server_submit; AFPS_ERR_INVALID_ARG
 * for memory that is not page-locked. */
int afps_server_submit_pinned(afps_server* srv, const float* h_xyz, int64_t N, uint64_t tag);

/* Withdraw the request with this tag (the oldest if several): a queued one
 * is removed at once; an admitted one is left out of the following steps and
 * its device memory and result slot are reclaimed once the steps already
 * launched have completed.  A cancelled request is never returned by
 * afps_server_poll.  AFPS_ERR_INVALID_ARG when no queued or admitted request
 * has the tag (or its result is already being returned). */
int afps_server_cancel(afps_server* srv, uint64_t tag);

/* One continuous-batching step (see above).  Returns the number of
 * single-level advances it made (requests times levels; 0 when idle), or a
 * negative error. */
int afps_server_step(afps_server* srv);

/* Move up to max_results finished requests into out; returns how many. */
int afps_server_poll(afps_server* srv, afps_server_result* out, int32_t max_results);

/* Counts of queued, in-flight (admitted, unfinished) requests and arena
 * bytes in use; any pointer may be NULL. */
int afps_server_stats(afps_server* srv, int64_t* queued, int64_t* inflight,
                      int64_t* arena_used);

/* Milliseconds since the server was created (the clock of the results). */
double afps_server_clock_ms(const afps_server* srv);

/* Wait for the server's device work and free everything it owns. */
void afps_server_destroy(afps_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* AFPS_H */
