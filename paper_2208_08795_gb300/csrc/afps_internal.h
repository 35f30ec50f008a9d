// afps_internal.h -- types shared by the host runtime (afps_api.cu) and the
// kernels (afps_kernels.cu, afps_gather.cu).  Not part of the public ABI.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace afps {

// One work item: one sector of one cloud (Sec. III-B).  Built on the host for
// batched calls; computed on the fly for a single cloud.
struct ItemDesc {
    int64_t src;    // global point index (into xyz) of the sector's first point
    int64_t dst;    // global output slot of the sector's first sample
    int32_t n;      // points in the sector
    int32_t c;      // samples taken from the sector
    int32_t first;  // sector offset of the first sample
    int32_t lo;     // sector's first point relative to its cloud (added to outputs)
    int32_t kl;     // NPDU window: points updated left of the sample
    int32_t kr;     // ... and right of it (kl = kr = 0 and no NPDU: whole sector)
    int32_t flags;  // ITEM_* bits
    int32_t pad;
};
static_assert(sizeof(ItemDesc) == 48, "ItemDesc layout");

// ItemDesc::flags
enum : int32_t { ITEM_FULL_FIRST = 1 };  // the first update reaches the whole sector

// A single cloud described by its parameters; items are its M sectors.
// A run of equal clouds (N points, C samples, M sectors each) stored back to
// back from point pt_off, their outputs back to back from out_off; a launch
// over it has (number of clouds) x M items.
// One cloud of a launch whose items are computed from per-cloud records.
struct CloudRec {
    int64_t pt_off;   // first point, in points from the xyz base
    int64_t out_off;  // first output, in elements from the output base
    int32_t N, C;
    int32_t pad[2];
};
static_assert(sizeof(CloudRec) == 32, "CloudRec layout");

struct SingleCloud {
    int64_t pt_off;
    int64_t out_off;
    int32_t N, C, M;
    int32_t kl, kr, flags;  // as in ItemDesc
    int32_t start_r;        // offset of start_idx inside its own sector
    int32_t wide;           // M * N >= 2^32: sector bounds in 64-bit arithmetic
    uint64_t m_magic;       // div_magic(M): x / M = high 64 bits of x * m_magic (x < 2^32)
    // Clouds at arbitrary offsets, of any N and C (the same M, window,
    // reading and start offset): a device array of records, one per cloud in
    // item order, replacing pt_off + b N, out_off + b C, N and C; nullptr for
    // equal clouds stored back to back.
    const CloudRec* clouds;
};

// Multiplier for unsigned division of 32-bit numerators by d >= 2:
// floor((2^64 - 1) / d) + 1 = ceil(2^64 / d) exceeds 2^64 / d by less than
// one, so x * m / 2^64 exceeds x / d by less than x / 2^64 < 2^-32 <= 1/d,
// which never reaches the next integer: the high word is floor(x / d).
// 0 for d < 2 (the caller divides instead).
inline uint64_t div_magic(int32_t d) {
    return d >= 2 ? ~0ull / (uint64_t)d + 1ull : 0ull;
}

enum Kind : int32_t { KIND_WARP = 0, KIND_CTA = 1, KIND_WIN = 2, KIND_WIN2 = 3 };

// A kernel variant.  KIND_WARP: one warp per item, W items per CTA.
// KIND_CTA: one CTA (CS == 1) or one cluster of CS CTAs per item, W warps
// per CTA.  P = points held per thread, in registers.  KIND_WIN (NPDU only):
// one warp per item, W items per CTA, distances in shared memory with cached
// row maxima; P = rows of 32 points a warp's buffer holds (sectors of up to
// 32 P points, P <= kWinMaxRows).  KIND_WIN2 (NPDU windows of at most 17
// points, literal reading): two items per warp, one per half-warp, W warps
// per CTA; P = rows of 16 points a half's buffer holds (sectors of up to 16 P
// points, P <= kWin2MaxRows).
struct Variant {
    int32_t kind;
    int32_t P;
    int32_t W;
    int32_t CS;
    int32_t occ;  // CTAs (or clusters) per SM for persistent grids; 0 = one per item
    int32_t skip; // NPDU: skip rows the window misses (uniform branch) instead of masking
};

struct LaunchArgs {
    const float* xyz;
    const ItemDesc* items;  // device table, or nullptr: use `single`
    SingleCloud single;
    int32_t n_items;
    int32_t* out;
    unsigned int* counter;  // dynamic work queue head (warp kind), or nullptr
    int* status;            // device error word (first error wins)
    uint64_t timeout_ns;
    uint32_t stall;         // fault injection (STALL_* bits)
    uint32_t npdu_skip;     // Variant::skip
    uint32_t host_resident; // points live in (mapped) host memory: plain loads only
    int32_t win_cap;        // KIND_WIN: points per warp buffer (32 P); KIND_WIN2: per half (16 P)
};

// LaunchArgs::stall bits (fault injection for tests of failure detection):
// the stage-in arms its barrier but issues no copy; in cluster kernels the
// last CTA of each cluster sends no exchange records.  Either way the
// bounded waits run out.
enum : uint32_t { STALL_COPY = 1u, STALL_EXCHANGE = 2u };

// Device error codes written to *status.
enum DeviceStatus : int {
    DEV_OK = 0,
    DEV_TIMEOUT_STAGE = 1,     // a stage-in bulk copy did not complete in time
    DEV_TIMEOUT_DRAIN = 2,     // ... nor within the second, draining wait
    DEV_TIMEOUT_EXCHANGE = 3,  // a cluster record exchange did not complete in time
    DEV_CHECK_FAILED = 4,      // a device-side check of the debug build failed
};

// KIND_WIN: largest number of 32-point rows per sector (lane l of the warp
// caches the maxima of rows l, l + 32, ..., up to kWinMaxRows / 32 of them).
constexpr int kWinMaxRows = 256;
// KIND_WIN2: largest number of 16-point rows per sector (8 slots of 16).
constexpr int kWin2MaxRows = 128;

// Points a variant can hold per item.
inline int64_t variant_capacity(const Variant& v) {
    if (v.kind == KIND_WIN2) return 16LL * v.P;
    return v.kind == KIND_CTA ? 32LL * v.W * v.P * v.CS : 32LL * v.P;
}

// Dynamic shared memory of a variant (bytes).
size_t variant_smem(const Variant& v);

// Whether the variant is compiled (P values, warp counts, cluster sizes).
bool variant_supported(const Variant& v);

// Launch the sector kernel for `v` on `stream`.  grid_hint = number of
// CTAs (warp kind) or clusters (CTA kind) to launch; the kernels stride over
// items when the grid is smaller than the item count.
cudaError_t launch_sector(const Variant& v, bool npdu, const LaunchArgs& a, int grid_hint,
                          cudaStream_t stream);

// Largest number of clusters of the variant that can be co-resident, or 0.
int max_active_clusters(const Variant& v);

// Chained-level gather (afps_gather_levels and the serving runtime).  All
// offsets are in elements of their arrays (points for xyz); -1 means "none"
// (identity frame indices on input, no output).
struct GatherDesc {
    int64_t in_xyz;     // first point of the cloud in in_xyz
    int64_t in_frame;   // first frame index of the cloud in in_frame, or -1
    int64_t sel;        // first sample in sel (indices relative to the cloud)
    int64_t out_xyz;    // first output point in out_xyz
    int64_t out_frame;  // first output entry in out_frame, or -1
    int64_t sel_frame;  // first output entry in sel_frame, or -1
    int32_t n;          // points in the cloud
    int32_t c;          // samples
};
cudaError_t launch_gather(const GatherDesc* d_descs, int32_t B, int32_t max_n,
                          const float* in_xyz, const int32_t* in_frame, const int32_t* sel,
                          float* out_xyz, int32_t* out_frame, int32_t* sel_frame,
                          cudaStream_t stream);
constexpr int32_t kGatherMaxPoints = 65536;

// Frames admitted by a serving step: from page-locked host memory (read by
// the kernel over the C2C link) into the device arena, one launch for all.
struct FrameCopy {
    const void* src;  // device-visible address of the host frame
    void* dst;        // arena address
    int64_t bytes;    // a multiple of 4
};
constexpr int kFrameCopyMax = 256;  // frames per launch (kernel-parameter batch)
struct FrameCopyBatch {
    int32_t n;
    int32_t pad;
    FrameCopy c[kFrameCopyMax];
};
cudaError_t launch_frame_copy(const FrameCopyBatch& batch, int64_t max_bytes, cudaStream_t stream);

// Coverage radius (afps_coverage_radius).
struct CoverageDesc {
    int64_t pt_off;   // first point of the cloud
    int64_t sel_off;  // first sample index
    int32_t n;        // points
    int32_t c;        // samples
};
cudaError_t launch_coverage(const CoverageDesc* d_descs, int32_t B, int32_t max_n,
                            const float* xyz, const int32_t* sel,
                            unsigned long long* max_bits, double* radius, cudaStream_t stream);

// Ball query (afps_ball_query).
struct GroupDesc {
    int64_t pt_off;   // first point of the cloud
    int64_t sel_off;  // first centroid (and output row)
    int32_t n;        // points
    int32_t c;        // centroids
};
cudaError_t launch_ball_query(const GroupDesc* d_descs, int32_t B, int32_t max_c,
                              const float* xyz, const int32_t* sel, float radius, int32_t K,
                              int32_t axis, int32_t* out, cudaStream_t stream);
// k nearest neighbours (afps_knn): one warp per centroid, 1 <= K <= 64.
cudaError_t launch_knn(const GroupDesc* d_descs, int32_t B, int32_t max_c, const float* xyz,
                       const int32_t* sel, int32_t K, int32_t axis, int32_t* out, float* dist2,
                       cudaStream_t stream);

// Sort by key (afps_sort_by_key): one cloud per CTA.
struct SortDesc {
    int64_t off;  // first point of the cloud
    int32_t n;    // points
    int32_t pad;
};
cudaError_t launch_sort(const SortDesc* d_descs, int32_t B, const float* xyz, int key,
                        uint32_t* keys_a, int32_t* idx_a, uint32_t* keys_b, int32_t* idx_b,
                        float* xyz_out, int32_t* perm, cudaStream_t stream);
// Large clouds: one thread-block cluster per cloud, the cloud in distributed
// shared memory (no scratch); clouds of up to sort_cluster_capacity() points.
cudaError_t launch_sort_cluster(const SortDesc* d_descs, int32_t B, int32_t max_n,
                                const float* xyz, int key, float* xyz_out, int32_t* perm,
                                cudaStream_t stream);
int sort_cluster_capacity();
// Clouds above this size go to the cluster sort (when they fit it).
constexpr int32_t kSortClusterMin = 4096;

}  // namespace afps

// ---- runtime functions over scattered clouds (afps_api.cu), for the server
struct afps_ctx;
namespace afps {
// Batched sampling of B clouds at arbitrary offsets of one xyz / output base.
// A second context on src's device, with its flags, timeout and tuned
// variants and a workspace of its own, sharing src's device status word (so
// afps_sync on src also reports its device errors): it lets work on another
// stream upload its tables without waiting for src's.  Destroy it with
// afps_destroy before src.
int clone_context(afps_ctx* src, afps_ctx** out);
// The last error message of `from`, for a caller that holds `to`.
void copy_error(afps_ctx* to, const afps_ctx* from);
int sample_scattered(afps_ctx* ctx, const float* xyz, int32_t B, const int64_t* pt_begin,
                     const int64_t* n_pts, const int32_t* C, const int32_t* M, const int32_t* K,
                     const int64_t* start, int32_t* out, const int64_t* out_begin,
                     cudaStream_t stream);
// Gather of B clouds described by host descriptors.
int gather_run(afps_ctx* ctx, const GatherDesc* descs, int32_t B, const float* in_xyz,
               const int32_t* in_frame, const int32_t* sel, float* out_xyz, int32_t* out_frame,
               int32_t* sel_frame, cudaStream_t stream);

}  // namespace afps
