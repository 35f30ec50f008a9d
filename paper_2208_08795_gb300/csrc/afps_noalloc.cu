// afps_noalloc.cu -- afps_sample_batched_noalloc: the batched sampler for
// callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc: code that runs inside another
// framework's memory pool or under a fixed device-memory budget, a plugin
// whose host application owns every allocation, or a real-time loop that must
// never take the allocator's locks or trigger an implicit device
// synchronisation.  For them this entry point needs no context and allocates
// no device memory (on the host heap only the first launch of each kernel
// variant on a device records the attributes set for it).  Its only scratch,
// the work-item table of the batched sector kernels plus a status word, is
// the file-scope array below, which every GPU that loads the library holds
// until the process exits.  The table goes up from a static host copy in
// pageable memory, so a call may wait for its stream, and a call on a
// capturing stream is refused.
//
// The sector kernels are the existing ones (afps_warp.cu, afps_cta.cu),
// launched without the persistent work queue: one warp, CTA or cluster per
// item, so no queue counter has to be zeroed.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <mutex>

#include "../../include/afps.h"
#include "afps_internal.h"
#include "afps_trace.h"

namespace {

constexpr int kMaxItems = AFPS_NOALLOC_MAX_ITEMS;
constexpr size_t kHeader = 256;  // status word, padded to the table's alignment
constexpr size_t kScratchBytes = kHeader + sizeof(afps::ItemDesc) * kMaxItems;
constexpr int kMaxDevices = 64;
// Launch classes: (variant, NPDU on/off) pairs na_variant can yield: 8 warp
// variants, CTA variants of 3-32 warps and clusters of 2-16 CTAs (53), each
// with and without NPDU, 106 in all.
constexpr int kMaxClasses = 128;

// The scratch: [status word | padding to 256 B | kMaxItems work items].
// In host code `g_noalloc_scratch` is a host-side stand-in, not a device
// address; its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

std::mutex g_mutex;                        // guards the two tables below
void* g_scratch_ptr[kMaxDevices];          // device address per device (set-up)
afps::ItemDesc g_host_items[kMaxItems];    // host staging of the item table

struct NaClass {
    afps::Variant v;
    bool npdu;
    int count;
    int first;
    int fill;
};

// Fixed launch policy (no tuning cache, no heap): smallest warp variant that
// holds the sector, else one CTA of 8 points per thread, else a cluster.
afps::Variant na_variant(int64_t n_max) {
    afps::Variant v{};
    v.CS = 1;
    if (n_max <= 512) {
        static const int kP[] = {1, 2, 3, 4, 6, 8, 12, 16};
        v.kind = afps::KIND_WARP;
        v.W = 4;
        for (int P : kP)
            if (32LL * P >= n_max) {
                v.P = P;
                break;
            }
        return v;
    }
    v.kind = afps::KIND_CTA;
    v.P = 8;
    v.skip = 1;
    if (n_max <= 8192) {
        v.W = (int)((n_max + 255) / 256);
        return v;
    }
    v.W = 32;
    v.CS = (int)((n_max + 8191) / 8192);
    return v;
}

bool same_variant(const afps::Variant& a, const afps::Variant& b) {
    return a.kind == b.kind && a.P == b.P && a.W == b.W && a.CS == b.CS && a.skip == b.skip;
}

// Sector rule of Sec. III-B: points [floor(sN/M), floor((s+1)N/M)), samples
// [floor(sC/M), floor((s+1)C/M)).  Validates one cloud; returns its largest
// sector and the start offset inside the start's sector.
int na_check(int64_t N, int32_t C, int32_t M, int32_t k, int64_t start, int64_t* n_max,
             int32_t* start_r) {
    if (N < 1 || N > INT32_MAX || C < 1 || (int64_t)C > N || M < 1 || M > C || k < 0 ||
        start < 0 || start >= N)
        return AFPS_ERR_INVALID_ARG;
    *n_max = 0;
    *start_r = 0;
    for (int64_t s = 0; s < M; ++s) {
        const int64_t lo = s * N / M, hi = (s + 1) * N / M;
        const int64_t c = (s + 1) * (int64_t)C / M - s * (int64_t)C / M;
        if (c > hi - lo) return AFPS_ERR_SECTOR_TOO_SMALL;
        if (hi - lo > *n_max) *n_max = hi - lo;
        if (start >= lo && start < hi) *start_r = (int32_t)(start - lo);
    }
    return *n_max > AFPS_MAX_SECTOR_POINTS ? AFPS_ERR_UNSUPPORTED : AFPS_OK;
}

// Device address of the scratch on the current device, looked up once per
// device (with that device current).
int na_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return AFPS_ERR_CUDA;
    }
    if (!g_scratch_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return AFPS_ERR_CUDA;
        }
        g_scratch_ptr[dev] = p;
    }
    *out = g_scratch_ptr[dev];
    return AFPS_OK;
}

}  // namespace

extern "C" int afps_sample_batched_noalloc(const float* d_xyz, const int64_t* h_pt_off,
                                           int32_t B, const int32_t* h_C, const int32_t* h_M,
                                           const int32_t* h_win, const int64_t* h_start,
                                           const int64_t* h_out_off, int32_t* d_out,
                                           void* stream) {
    AFPS_TRACE("afps_sample_batched_noalloc");
    if (!d_xyz || !d_out || B < 1 || !h_pt_off || !h_C || !h_M || !h_win || !h_start ||
        !h_out_off)
        return AFPS_ERR_INVALID_ARG;
    if (reinterpret_cast<uintptr_t>(d_xyz) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4 ||
        h_pt_off[0] < 0 || h_out_off[0] < 0)
        return AFPS_ERR_INVALID_ARG;
    // not under stream capture: the table's upload from the static host copy
    // would be recorded, and replays would read whatever a later call left there
    {
        cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
        if (cudaStreamIsCapturing(static_cast<cudaStream_t>(stream), &cs) != cudaSuccess) {
            cudaGetLastError();
            return AFPS_ERR_INVALID_ARG;
        }
        if (cs != cudaStreamCaptureStatusNone) return AFPS_ERR_INVALID_ARG;
    }

    // pass 1: validate, size the item table, form launch classes
    NaClass cls[kMaxClasses];
    int n_cls = 0;
    int64_t total = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t N = h_pt_off[b + 1] - h_pt_off[b];
        if (h_out_off[b + 1] - h_out_off[b] < (int64_t)h_C[b]) return AFPS_ERR_INVALID_ARG;
        int64_t n_max;
        int32_t start_r;
        const int rc = na_check(N, h_C[b], h_M[b], h_win[b], h_start[b], &n_max, &start_r);
        if (rc != AFPS_OK) return rc;
        total += h_M[b];
        if (total > kMaxItems) return AFPS_ERR_SCRATCH_TOO_SMALL;
        const afps::Variant v = na_variant(n_max);
        const bool npdu = h_win[b] > 0;
        int c = 0;
        while (c < n_cls && !(cls[c].npdu == npdu && same_variant(cls[c].v, v))) ++c;
        if (c == n_cls) {
            if (n_cls == kMaxClasses) return AFPS_ERR_UNSUPPORTED;
            cls[n_cls++] = NaClass{v, npdu, 0, 0, 0};
        }
        cls[c].count += h_M[b];
    }
    for (int c = 0, first = 0; c < n_cls; ++c) {
        cls[c].first = first;
        cls[c].fill = first;
        first += cls[c].count;
    }

    std::lock_guard<std::mutex> lock(g_mutex);
    void* scratch = nullptr;
    int rc = na_scratch(&scratch);
    if (rc != AFPS_OK) return rc;

    // pass 2: write the items class-major into the static host staging
    for (int32_t b = 0; b < B; ++b) {
        const int64_t N = h_pt_off[b + 1] - h_pt_off[b];
        const int32_t C = h_C[b], M = h_M[b];
        int64_t n_max;
        int32_t start_r;
        na_check(N, C, M, h_win[b], h_start[b], &n_max, &start_r);
        const afps::Variant v = na_variant(n_max);
        const bool npdu = h_win[b] > 0;
        int c = 0;
        while (!(cls[c].npdu == npdu && same_variant(cls[c].v, v))) ++c;
        const int32_t k = (int32_t)(h_win[b] < 4LL * AFPS_MAX_SECTOR_POINTS
                                        ? h_win[b]
                                        : 4LL * AFPS_MAX_SECTOR_POINTS);
        for (int64_t s = 0; s < M; ++s) {
            afps::ItemDesc& d = g_host_items[cls[c].fill++];
            const int64_t lo = s * N / M, hi = (s + 1) * N / M;
            const int64_t o0 = s * (int64_t)C / M, o1 = (s + 1) * (int64_t)C / M;
            d.src = h_pt_off[b] + lo;
            d.dst = h_out_off[b] + o0;
            d.n = (int32_t)(hi - lo);
            d.c = (int32_t)(o1 - o0);
            d.first = start_r < d.n - 1 ? start_r : d.n - 1;
            d.lo = (int32_t)lo;
            d.kl = k / 2;  // the default NPDU window: k neighbours and the sample
            d.kr = k - k / 2;
            d.flags = 0;
            d.pad = 0;
        }
    }

    // the status word must start at zero; the table is overwritten in full
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    unsigned char* base = static_cast<unsigned char*>(scratch);
    afps::ItemDesc* d_items = reinterpret_cast<afps::ItemDesc*>(base + kHeader);
    if (cudaMemsetAsync(base, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemcpyAsync(d_items, g_host_items, (size_t)total * sizeof(afps::ItemDesc),
                        cudaMemcpyHostToDevice, st) != cudaSuccess) {
        cudaGetLastError();
        return AFPS_ERR_CUDA;
    }
    for (int c = 0; c < n_cls; ++c) {
        afps::LaunchArgs a{};
        a.xyz = d_xyz;
        a.items = d_items + cls[c].first;
        a.n_items = cls[c].count;
        a.out = d_out;
        a.counter = nullptr;
        a.status = reinterpret_cast<int*>(base);
        a.timeout_ns = 2000000000ull;
        a.stall = 0;
        a.npdu_skip = cls[c].v.skip ? 1u : 0u;
        const int grid = cls[c].v.kind == afps::KIND_WARP
                             ? (cls[c].count + cls[c].v.W - 1) / cls[c].v.W
                             : cls[c].count;
        if (afps::launch_sector(cls[c].v, cls[c].npdu, a, grid, st) != cudaSuccess) {
            cudaGetLastError();
            return AFPS_ERR_CUDA;
        }
    }
    return AFPS_OK;
}
