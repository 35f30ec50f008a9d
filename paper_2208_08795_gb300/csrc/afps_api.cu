// afps_api.cu -- the C ABI of include/afps.h: argument checks, the sector
// plan (Sec. III-B), kernel-variant choice, the batched work-item table,
// CUDA-graph replay, the autotuner and device-error reporting.
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/afps.h"
#include "afps_internal.h"
#include "afps_trace.h"

using afps::ItemDesc;
using afps::LaunchArgs;
using afps::SingleCloud;
using afps::Variant;

namespace {

constexpr uint64_t kDefaultTimeoutNs = 2000000000ull;
constexpr size_t kMaxGraphs = 512;  // cached graphs per context (least recently used evicted)
constexpr size_t kMaxPlans = 256;   // cached batch plans per context (cleared when full)
constexpr int kStageSlots = 16;  // pinned upload buffers in flight

// ---------------------------------------------------------------- buffers
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    // Grows to at least twice its size: each growth frees (which waits for
    // the device) and allocates, so a slowly rising need must not pay it often.
    cudaError_t reserve(size_t want) {
        if (want <= bytes) return cudaSuccess;
        const size_t cap = std::max({want, 2 * bytes, (size_t)4096});
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, cap);
        if (e == cudaSuccess) bytes = cap;
        return e;
    }
    void release() {
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
    }
};

struct HostBuf {
    void* p = nullptr;
    size_t bytes = 0;
    // Grows to at least twice its size (page-locked allocations are slow).
    cudaError_t reserve(size_t want) {
        if (want <= bytes) return cudaSuccess;
        const size_t cap = std::max({want, 2 * bytes, (size_t)4096});
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMallocHost(&p, cap);
        if (e == cudaSuccess) bytes = cap;
        return e;
    }
    void release() {
        if (p) cudaFreeHost(p);
        p = nullptr;
        bytes = 0;
    }
};

// One launch class of a batched call: items that share a kernel variant.
struct ClassPlan {
    bool npdu = false;
    int64_t n_max = 0;
    int32_t c_max = 0;
    Variant v{};
    size_t first = 0;  // first item in the concatenated table
    size_t count = 0;
    // every cloud of the class has the same N, C, M, window and start, and
    // they are stored back to back: the kernel computes its items
    bool uniform = false;
    // items computed from per-cloud records, which start at record
    // cloud_first of BatchPlan::clouds (-1: equal clouds back to back)
    int64_t cloud_first = -1;
    bool merged = false;  // several shape classes in one launch (window kernels)
    bool narrow = true;   // every item's window has at most 17 points, read literally
    afps::SingleCloud single{};
    const afps::SingleCloud* run() const { return uniform ? &single : nullptr; }
};

struct BatchPlan {
    std::vector<ItemDesc> items;  // class-major
    std::vector<ClassPlan> classes;
    std::vector<afps::CloudRec> clouds;  // per-cloud records of the record classes
};

struct GraphEntry {
    cudaGraphExec_t exec = nullptr;
    DevBuf items;
    DevBuf counters;
    DevBuf xyz, out;  // device staging of a host-buffer graph
    int64_t kernels = 0;
    uint64_t last_use = 0;
};

}  // namespace

struct afps_ctx {
    int device = 0;
    uint32_t flags = 0;
    uint64_t timeout_ns = kDefaultTimeoutNs;
    std::string tune_path;
    int num_sms = 0;
    int* d_status = nullptr;
    bool status_borrowed = false;  // d_status belongs to another context (clone_context)
    std::string last_error;
    cudaEvent_t ev_done = nullptr;    // last device work that used the shared workspace
    cudaStream_t capture = nullptr;   // private stream for graph capture
    DevBuf items, counters, xyz_stage, out_stage, sort_scratch, cov_scratch;
    HostBuf stage[kStageSlots];         // pinned upload ring
    cudaEvent_t stage_ev[kStageSlots] = {};  // last copy out of each slot
    int stage_next = 0;
    std::unordered_map<std::string, GraphEntry> graphs;
    std::unordered_map<std::string, BatchPlan> plans;  // batched calls without graphs
    std::unordered_set<std::string> checked;  // argument sets whose classes are tuned (AUTOTUNE)
    std::map<std::string, Variant> tuned;
    int64_t launches = 0;
    uint64_t tick = 0;
};

namespace {

int fail(afps_ctx* ctx, int code, const std::string& msg) {
    if (ctx) ctx->last_error = msg;
    return code;
}

int cuda_fail(afps_ctx* ctx, cudaError_t e, const char* what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();  // clear a sticky launch error so the context stays usable
    return fail(ctx, e == cudaErrorMemoryAllocation ? AFPS_ERR_NO_MEMORY : AFPS_ERR_CUDA, m);
}

// Growth of a workspace buffer of the context (device or page-locked).
// AFPS_FLAG_TEST_FAIL_ALLOC makes every growth fail as on an exhausted
// device (fault injection).
template <class Buf>
cudaError_t grow(afps_ctx* ctx, Buf& b, size_t want) {
    if (want > b.bytes && (ctx->flags & AFPS_FLAG_TEST_FAIL_ALLOC)) return cudaErrorMemoryAllocation;
    return b.reserve(want);
}

#define AFPS_CUDA(ctx, call)                                   \
    do {                                                       \
        cudaError_t e_ = (call);                               \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
    }
};

// ---------------------------------------------------------------- sectors
// Sector s of a cloud (Sec. III-B): points [floor(sN/M), floor((s+1)N/M)),
// output slots [floor(sC/M), floor((s+1)C/M)).
inline int64_t sec_lo(int64_t N, int64_t M, int64_t s) { return s * N / M; }
inline int64_t sec_off(int64_t C, int64_t M, int64_t s) { return s * C / M; }

// A window of k >= 2n covers the whole sector wherever the sample lies, so
// clamping k there changes no result and keeps p + k in int32 on the device.
inline int32_t device_window(int32_t k) {
    return (int32_t)std::min<int64_t>(k, 4LL * AFPS_MAX_SECTOR_POINTS);
}

// Window extents and item flags of the NPDU reading `method` (afps.h).
void window_sides(int32_t k, uint32_t method, ItemDesc& d) {
    const int32_t kk = device_window(k);
    if (kk > 0 && (method & AFPS_METHOD_WINDOW_HAS_SAMPLE)) {
        d.kl = (kk - 1) / 2;
        d.kr = (kk - 1) - (kk - 1) / 2;
    } else {
        d.kl = kk / 2;
        d.kr = kk - kk / 2;
    }
    d.flags = (kk > 0 && (method & AFPS_METHOD_FULL_FIRST_PASS)) ? afps::ITEM_FULL_FIRST : 0;
}

struct CloudCheck {
    int code = AFPS_OK;
    std::string msg;
    int64_t n_max = 0;
    int32_t c_max = 0;
    int32_t start_r = 0;
};

// (The message streams are built on the error paths only: constructing one
// costs about a microsecond, once per cloud of every call.)
CloudCheck check_cloud(int64_t N, int32_t C, int32_t M, int32_t k, int64_t start) {
    CloudCheck r;
    if (N < 1 || N > INT32_MAX || C < 1 || (int64_t)C > N || M < 1 || M > C || k < 0 ||
        start < 0 || start >= N) {
        std::ostringstream os;
        os << "invalid arguments: N=" << N << " C=" << C << " M=" << M << " k=" << k
           << " start=" << start << " (need 1<=C<=N<2^31, 1<=M<=C, k>=0, 0<=start<N)";
        r.code = AFPS_ERR_INVALID_ARG;
        r.msg = os.str();
        return r;
    }
    int64_t s0 = -1;
    for (int64_t s = 0; s < M; ++s) {
        const int64_t lo = sec_lo(N, M, s), hi = sec_lo(N, M, s + 1);
        const int64_t c = sec_off(C, M, s + 1) - sec_off(C, M, s);
        if (c > hi - lo) {
            std::ostringstream os;
            os << "sector " << s << " has " << (hi - lo) << " points but " << c
               << " samples (N=" << N << " C=" << C << " M=" << M << ")";
            r.code = AFPS_ERR_SECTOR_TOO_SMALL;
            r.msg = os.str();
            return r;
        }
        r.n_max = std::max(r.n_max, hi - lo);
        r.c_max = std::max<int32_t>(r.c_max, (int32_t)c);
        if (start >= lo && start < hi) s0 = s;
    }
    r.start_r = (int32_t)(start - sec_lo(N, M, s0));
    if (r.n_max > AFPS_MAX_SECTOR_POINTS) {
        std::ostringstream os;
        os << "sector of " << r.n_max << " points exceeds AFPS_MAX_SECTOR_POINTS ("
           << AFPS_MAX_SECTOR_POINTS << ")";
        r.code = AFPS_ERR_UNSUPPORTED;
        r.msg = os.str();
    }
    return r;
}

// ---------------------------------------------------------------- variants
const int kWarpP[] = {1, 2, 3, 4, 6, 8, 12, 16, 24, 32};
const int kCtaP[] = {2, 4, 8, 16};

// Window-kernel variant for NPDU sectors of up to n_max points: a buffer of
// exactly the rows needed, and the most warps per CTA (a power of two, at
// most 8) whose buffers fit in 64 KB, so that several CTAs share an SM.
// lean (Variant::skip): the round form with the fewest instructions, for
// classes with many sectors; otherwise the one with the shortest chain.
Variant win_variant(int64_t n_max, int W = 0, bool lean = false) {
    Variant v{};
    v.kind = afps::KIND_WIN;
    v.P = (int)((n_max + 31) / 32);
    v.CS = 1;
    v.skip = lean ? 1 : 0;
    if (W > 0) {
        v.W = W;
        return v;
    }
    const int64_t per_warp = 16 * 32 * (int64_t)v.P + 16;
    v.W = 8;
    while (v.W > 1 && v.W * per_warp > 64 * 1024) v.W /= 2;
    return v;
}

// Pair-kernel variant (two sectors per warp, 16-point rows) for narrow
// NPDU windows and sectors of up to n_max points: W as for win_variant.
Variant win2_variant(int64_t n_max, int W = 0) {
    Variant v{};
    v.kind = afps::KIND_WIN2;
    v.P = (int)((n_max + 15) / 16);
    v.CS = 1;
    if (W > 0) {
        v.W = W;
        return v;
    }
    const int64_t per_warp = 2 * (16 * 16 * (int64_t)v.P + 16);
    v.W = 8;
    while (v.W > 1 && v.W * per_warp > 64 * 1024) v.W /= 2;
    return v;
}

// Whether NPDU sectors of up to n_max points go to the window kernel by
// default: above 64 points (two rows per lane in the register kernel, where
// its full rescan is as cheap as the row cache) and up to its capacity.
bool win_default(int64_t n_max) { return n_max > 64 && n_max <= 32LL * afps::kWinMaxRows; }

// Default variant for sectors of up to n_max points; `many`: the class has
// more sectors than the GPU runs at once several times over (its time is
// then set by the instructions it issues, not by one sector's chain).
Variant default_variant(int64_t n_max, bool npdu, bool many = false) {
    if (npdu && win_default(n_max)) return win_variant(n_max, 0, many);
    Variant v{};
    v.CS = 1;
    v.occ = 0;
    if (n_max <= 512) {
        v.kind = afps::KIND_WARP;
        for (int P : kWarpP)
            if (32LL * P >= n_max) {
                v.P = P;
                break;
            }
        v.W = v.P <= 4 ? 8 : 4;
        return v;
    }
    v.kind = afps::KIND_CTA;
    v.skip = 1;
    if (n_max <= 4096) {
        v.P = 4;
        v.W = (int)((n_max + 127) / 128);
        return v;
    }
    if (n_max <= 8192) {
        v.P = 8;
        v.W = (int)((n_max + 255) / 256);
        return v;
    }
    v.P = 8;
    v.W = 16;
    v.CS = (int)((n_max + 4095) / 4096);
    if (v.CS > 16) {
        v.W = 32;
        v.CS = (int)((n_max + 8191) / 8192);
    }
    return v;
}

// Every variant the autotuner tries for sectors of up to n_max points (with
// and without the NPDU row skip when the class uses NPDU).
std::vector<Variant> candidate_variants(int64_t n_max, bool npdu, bool narrow = false) {
    std::vector<Variant> out;
    if (n_max <= 1024) {
        for (int P : kWarpP) {
            if (32LL * P < n_max) continue;
            for (int W : {2, 4, 8}) out.push_back(Variant{afps::KIND_WARP, P, W, 1, 0, 0});
            break;  // the smallest P that fits: larger P only adds padding
        }
    }
    for (int P : kCtaP) {
        const int64_t W = (n_max + 32LL * P - 1) / (32LL * P);
        if (W >= 1 && W <= 32 && n_max > 64)
            out.push_back(Variant{afps::KIND_CTA, P, (int)W, 1, 0, 0});
    }
    if (n_max > 2048) {
        for (int P : {4, 8, 16})
            for (int W : {4, 8, 16, 32}) {
                const int64_t CS = (n_max + 32LL * W * P - 1) / (32LL * W * P);
                if (CS >= 2 && CS <= 16) out.push_back(Variant{afps::KIND_CTA, P, W, (int)CS, 0, 0});
            }
    }
    std::vector<Variant> ok;
    for (const Variant& v : out) {
        if (!afps::variant_supported(v) || afps::variant_capacity(v) < n_max) continue;
        ok.push_back(v);
        if (npdu) {
            Variant s = v;
            s.skip = 1;
            ok.push_back(s);
        }
    }
    if (npdu && win_default(n_max))  // (up to 64 points the register kernels win)
        for (int W : {1, 2, 4, 8}) {
            for (bool lean : {false, true}) {
                const Variant v = win_variant(n_max, W, lean);
                if (afps::variant_supported(v)) ok.push_back(v);
            }
            const Variant v2 = win2_variant(n_max, W);
            if (narrow && afps::variant_supported(v2) && afps::variant_capacity(v2) >= n_max)
                ok.push_back(v2);
        }
    return ok;
}

std::string class_key(bool npdu, int64_t n_max, int32_t c_max, size_t items) {
    size_t b = 1;
    while (b < items) b <<= 1;
    std::ostringstream os;
    os << (npdu ? "npdu" : "full") << ":n" << n_max << ":c" << c_max << ":i" << b;
    return os.str();
}

Variant choose_variant(const afps_ctx* ctx, bool npdu, int64_t n_max, int32_t c_max,
                       size_t items, bool narrow = false) {
    auto it = ctx->tuned.find(class_key(npdu, n_max, c_max, items));
    const bool windows = it != ctx->tuned.end() &&
                         (it->second.kind == afps::KIND_WIN || it->second.kind == afps::KIND_WIN2);
    if (it != ctx->tuned.end() && afps::variant_capacity(it->second) >= n_max &&
        afps::variant_supported(it->second) && (npdu || !windows) &&
        (narrow || it->second.kind != afps::KIND_WIN2))
        return it->second;
    return default_variant(n_max, npdu, items >= 8 * (size_t)std::max(ctx->num_sms, 1));
}

std::string describe(const Variant& v) {
    std::ostringstream os;
    if (v.kind == afps::KIND_WARP)
        os << "warp P=" << v.P << " W=" << v.W;
    else if (v.kind == afps::KIND_WIN)
        os << "win P=" << v.P << " W=" << v.W << (v.skip ? " lean" : "");
    else if (v.kind == afps::KIND_WIN2)
        os << "pair P=" << v.P << " W=" << v.W;
    else if (v.CS > 1)
        os << "cluster P=" << v.P << " W=" << v.W << " CS=" << v.CS;
    else
        os << "cta P=" << v.P << " W=" << v.W;
    if (v.skip && v.kind != afps::KIND_WIN && v.kind != afps::KIND_WIN2) os << " skip";
    return os.str();
}

}  // namespace

namespace {

// ---------------------------------------------------------------- launching
// Grid for `count` items of variant v: one CTA per W items (warp kind) or
// one CTA / cluster per item, capped at what can be co-resident, in which
// case the kernels stride over the remaining items (persistent launch).
int grid_for(const Variant& v, size_t count) {
    static std::map<std::tuple<int, int, int, int>, int> cache;
    auto key = std::make_tuple(v.kind, v.P, v.W, v.CS);
    auto it = cache.find(key);
    int cap;
    if (it == cache.end()) {
        cap = afps::max_active_clusters(v);
        cache[key] = cap;
    } else {
        cap = it->second;
    }
    const size_t per_cta = v.kind == afps::KIND_WIN2 ? 2 * (size_t)v.W : (size_t)v.W;
    size_t want = v.kind != afps::KIND_CTA ? (count + per_cta - 1) / per_cta : count;
    if (cap > 0 && want > (size_t)cap) want = (size_t)cap;
    return (int)std::max<size_t>(want, 1);
}

// Fault-injection bits of the sector kernels for the context's flags.
uint32_t stall_bits(uint32_t flags) {
    return ((flags & AFPS_FLAG_TEST_STALL_COPY) ? afps::STALL_COPY : 0u) |
           ((flags & AFPS_FLAG_TEST_STALL_EXCHANGE) ? afps::STALL_EXCHANGE : 0u);
}

// Whether a launch of `count` items of variant v takes its items from a
// dynamic work queue: warp-per-item kernels whose grid is capped below one
// warp per item (persistent launch); otherwise items map to warps 1:1.
bool uses_queue(const Variant& v, size_t count) {
    const size_t per_cta = v.kind == afps::KIND_WIN2 ? 2 * (size_t)v.W : (size_t)v.W;
    return v.kind != afps::KIND_CTA && (size_t)grid_for(v, count) * per_cta < count;
}

// Work-queue counters start at zero and every launch leaves its counter at
// zero (the warp that draws the last ticket resets it), so a counter buffer
// is cleared only when it is allocated.
int grow_counters(afps_ctx* ctx, DevBuf& b, size_t n, cudaStream_t stream) {
    const size_t want = n * sizeof(unsigned int);
    if (want <= b.bytes) return AFPS_OK;
    AFPS_CUDA(ctx, grow(ctx, b, want));
    AFPS_CUDA(ctx, cudaMemsetAsync(b.p, 0, b.bytes, stream));
    return AFPS_OK;
}

int launch_class(afps_ctx* ctx, const Variant& v, bool npdu, const ItemDesc* d_items,
                 size_t count, unsigned int* d_counter, const float* xyz, int32_t* out,
                 cudaStream_t stream, bool host_resident = false,
                 const afps::SingleCloud* run = nullptr) {
    LaunchArgs a{};
    a.xyz = xyz;
    a.items = run ? nullptr : d_items;
    if (run) a.single = *run;
    a.n_items = (int32_t)count;
    a.out = out;
    const int grid = grid_for(v, count);
    a.counter = uses_queue(v, count) ? d_counter : nullptr;  // left at zero by the kernel
    a.status = ctx->d_status;
    a.timeout_ns = ctx->timeout_ns;
    a.stall = stall_bits(ctx->flags);
    a.npdu_skip = v.skip ? 1u : 0u;
    a.host_resident = host_resident ? 1u : 0u;
    cudaError_t e = afps::launch_sector(v, npdu, a, grid, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "sector kernel launch");
    ctx->launches += 1;
    return AFPS_OK;
}

// Size class of a sector: the warp capacities up to 512 points, then powers
// of two.  Clouds of one class share a kernel variant in a batched call.
int64_t size_bucket(int64_t n_max) {
    if (n_max <= 512) {
        for (int P : kWarpP)
            if (32LL * P >= n_max) return 32LL * P;
    }
    int64_t b = 1024;
    while (b < n_max) b <<= 1;
    return b;
}

// Cloud b: n_pts[b] points from point pt_begin[b] of the xyz base, C[b]
// indices written from out_begin[b] of the output base (out_cap[b] slots).
// Work of an item, for largest-first ordering of a class's queue.
int64_t item_cost(const ItemDesc& d, bool npdu) {
    return npdu ? (int64_t)d.c * (d.kl + d.kr + 1 + d.n / 32) : (int64_t)d.c * d.n;
}

// Consecutive table classes whose variants are window kernels of the same
// kind run as one launch: the buffer and the template (row-maximum slots per
// lane) for the largest sectors hold the smaller ones, and one dynamic queue
// over all of them (largest work first) leaves a shorter tail than launches
// one after the other.  The items of consecutive classes are contiguous in
// the table.
void merge_window_classes(BatchPlan& plan) {
    std::vector<ClassPlan> out;
    for (const ClassPlan& cp : plan.classes) {
        if (!out.empty()) {
            ClassPlan& last = out.back();
            const bool windows = last.v.kind == afps::KIND_WIN || last.v.kind == afps::KIND_WIN2;
            if (!last.uniform && !cp.uniform && last.npdu && cp.npdu && windows &&
                last.v.kind == cp.v.kind && last.first + last.count == cp.first) {
                if (cp.v.P > last.v.P) last.v = cp.v;
                last.count += cp.count;
                last.n_max = std::max(last.n_max, cp.n_max);
                last.c_max = std::max(last.c_max, cp.c_max);
                last.narrow = last.narrow && cp.narrow;
                last.merged = true;  // re-sorted below
                continue;
            }
        }
        out.push_back(cp);
    }
    for (const ClassPlan& cp : out)
        if (cp.merged)
            std::stable_sort(plan.items.begin() + cp.first,
                             plan.items.begin() + cp.first + cp.count,
                             [](const ItemDesc& x, const ItemDesc& y) {
                                 return item_cost(x, true) > item_cost(y, true);
                             });
    plan.classes.swap(out);
}

int build_plan(afps_ctx* ctx, int32_t B, const int64_t* pt_begin, const int64_t* n_pts,
               const int64_t* out_begin, const int64_t* out_cap, const int32_t* C,
               const int32_t* M, const int32_t* K, const int64_t* start, BatchPlan& plan,
               const uint32_t* method = nullptr, bool merge = true, bool scatter = false) {
    if (B < 1 || !pt_begin || !n_pts || !out_begin || !out_cap || !C || !M || !K || !start)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "batched call: B < 1 or a NULL host array");
    struct Member {
        int32_t b;
        CloudCheck chk;
    };
    std::map<std::pair<int, int64_t>, std::vector<Member>> groups;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t N = n_pts[b];
        if (pt_begin[b] < 0 || out_begin[b] < 0) {
            std::ostringstream os;
            os << "cloud " << b << ": negative point or output offset";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        if (out_cap[b] < (int64_t)C[b]) {
            std::ostringstream os;
            os << "cloud " << b << ": output range " << out_cap[b] << " is smaller than C=" << C[b];
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        CloudCheck chk = check_cloud(N, C[b], M[b], K[b], start[b]);
        if (chk.code != AFPS_OK) {
            std::ostringstream os;
            os << "cloud " << b << ": " << chk.msg;
            return fail(ctx, chk.code, os.str());
        }
        if (method && method[b] > AFPS_METHOD_ALL) {
            std::ostringstream os;
            os << "cloud " << b << ": unknown method bits " << method[b];
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        groups[{K[b] > 0 ? 1 : 0, size_bucket(chk.n_max)}].push_back(Member{b, chk});
    }
    plan.items.clear();
    plan.classes.clear();
    plan.clouds.clear();
    for (auto& g : groups) {
        ClassPlan cp;
        cp.npdu = g.first.first == 1;
        cp.first = plan.items.size();
        // a run of equal clouds stored back to back: items computed on the device
        {
            const Member& m0 = g.second.front();
            const int32_t b0 = m0.b;
            const uint32_t meth0 = method ? method[b0] : 0u;
            bool same = true;    // every cloud of the class has the same M, window,
                                 // reading and start offset ...
            bool equal = true;   // ... the same N and C ...
            bool packed = true;  // ... and they lie back to back
            int64_t wide_mn = 0;  // largest M * N
            for (size_t j = 0; j < g.second.size() && same; ++j) {
                const Member& m = g.second[j];
                const int32_t b = m.b;
                same = M[b] == M[b0] && K[b] == K[b0] && (method ? method[b] : 0u) == meth0 &&
                       m.chk.start_r == m0.chk.start_r && n_pts[b] <= INT32_MAX;
                equal = equal && n_pts[b] == n_pts[b0] && C[b] == C[b0];
                packed = packed && pt_begin[b] == pt_begin[b0] + (int64_t)j * n_pts[b0] &&
                         out_begin[b] == out_begin[b0] + (int64_t)j * C[b0];
                wide_mn = std::max(wide_mn, (int64_t)M[b] * n_pts[b]);
            }
            // clouds elsewhere or of different sizes: one record per cloud
            // instead of M table entries (worth it from two clouds on)
            const bool records = scatter && !(equal && packed) && g.second.size() >= 2;
            if (same && ((equal && packed) || records)) {
                ItemDesc w{};
                window_sides(K[b0], meth0, w);
                cp.uniform = true;
                int64_t n_max = 0;
                int32_t c_max = 0;
                if (records) {
                    // largest clouds first: the queue's items then come in
                    // about the longest-processing-time order
                    std::vector<Member> order(g.second);
                    std::stable_sort(order.begin(), order.end(),
                                     [&](const Member& x, const Member& y) {
                                         return (int64_t)C[x.b] * n_pts[x.b] >
                                                (int64_t)C[y.b] * n_pts[y.b];
                                     });
                    cp.cloud_first = (int64_t)plan.clouds.size();
                    for (const Member& m : order) {
                        afps::CloudRec r{};
                        r.pt_off = pt_begin[m.b];
                        r.out_off = out_begin[m.b];
                        r.N = (int32_t)n_pts[m.b];
                        r.C = C[m.b];
                        plan.clouds.push_back(r);
                        n_max = std::max(n_max, m.chk.n_max);
                        c_max = std::max(c_max, m.chk.c_max);
                    }
                } else {
                    n_max = m0.chk.n_max;
                    c_max = m0.chk.c_max;
                }
                cp.single.pt_off = records ? 0 : pt_begin[b0];
                cp.single.out_off = records ? 0 : out_begin[b0];
                cp.single.N = (int32_t)n_pts[b0];
                cp.single.C = C[b0];
                cp.single.M = M[b0];
                cp.single.kl = w.kl;
                cp.single.kr = w.kr;
                cp.single.flags = w.flags;
                cp.single.start_r = m0.chk.start_r;
                cp.single.wide = wide_mn > (int64_t)UINT32_MAX ? 1 : 0;
                cp.single.m_magic = afps::div_magic(M[b0]);
                cp.n_max = n_max;
                cp.c_max = c_max;
                cp.count = g.second.size() * (size_t)M[b0];
                cp.narrow = w.kl + w.kr <= 16 && !(w.flags & afps::ITEM_FULL_FIRST);
                cp.v = choose_variant(ctx, cp.npdu, cp.n_max, cp.c_max, cp.count, cp.narrow);
                plan.classes.push_back(cp);
                continue;
            }
        }
        for (const Member& m : g.second) {
            const int32_t b = m.b;
            const int64_t N = n_pts[b];
            cp.n_max = std::max(cp.n_max, m.chk.n_max);
            cp.c_max = std::max(cp.c_max, m.chk.c_max);
            int64_t hi = 0, o1 = 0;  // each sector's end is the next one's start
            for (int64_t s = 0; s < M[b]; ++s) {
                const int64_t lo = hi, o0 = o1;
                hi = sec_lo(N, M[b], s + 1);
                o1 = sec_off(C[b], M[b], s + 1);
                ItemDesc d{};
                d.src = pt_begin[b] + lo;
                d.dst = out_begin[b] + o0;
                d.n = (int32_t)(hi - lo);
                d.c = (int32_t)(o1 - o0);
                d.first = std::min<int32_t>(m.chk.start_r, d.n - 1);
                d.lo = (int32_t)lo;
                window_sides(K[b], method ? method[b] : 0u, d);
                cp.narrow = cp.narrow && d.kl + d.kr <= 16 && !(d.flags & afps::ITEM_FULL_FIRST);
                plan.items.push_back(d);
            }
        }
        cp.count = plan.items.size() - cp.first;
        // largest work first (longest-processing-time order for the queue),
        // equal costs in table order; the keys are sorted, not the entries
        const bool npdu = cp.npdu;
        std::vector<std::pair<int64_t, uint32_t>> key(cp.count);
        bool ordered = true;
        for (size_t j = 0; j < cp.count; ++j) {
            key[j] = {-item_cost(plan.items[cp.first + j], npdu), (uint32_t)j};
            ordered = ordered && (j == 0 || key[j].first >= key[j - 1].first);
        }
        if (!ordered) {
            std::sort(key.begin(), key.end());
            std::vector<ItemDesc> sorted(cp.count);
            for (size_t j = 0; j < cp.count; ++j) sorted[j] = plan.items[cp.first + key[j].second];
            std::copy(sorted.begin(), sorted.end(), plan.items.begin() + cp.first);
        }
        cp.v = choose_variant(ctx, cp.npdu, cp.n_max, cp.c_max, cp.count, cp.narrow);
        plan.classes.push_back(cp);
    }
    if (merge) merge_window_classes(plan);
    return AFPS_OK;
}

// Copy `bytes` of host data into the device buffer `dst` on `stream`, through
// the next slot of the pinned upload ring (waiting only for that slot's
// previous copy, kStageSlots uploads ago).  Device work that used the
// workspace earlier, possibly on another stream, is ordered before the copy.
// A second part (src2, bytes2) goes right after the first in the same copy.
int upload(afps_ctx* ctx, DevBuf& dst, const void* src, size_t bytes, cudaStream_t stream,
           const void* src2 = nullptr, size_t bytes2 = 0) {
    const int s = ctx->stage_next;
    ctx->stage_next = (s + 1) % kStageSlots;
    const size_t total = bytes + bytes2;
    AFPS_CUDA(ctx, cudaEventSynchronize(ctx->stage_ev[s]));
    AFPS_CUDA(ctx, grow(ctx, ctx->stage[s], total));
    AFPS_CUDA(ctx, grow(ctx, dst, total));
    if (bytes) memcpy(ctx->stage[s].p, src, bytes);
    if (bytes2) memcpy(static_cast<char*>(ctx->stage[s].p) + bytes, src2, bytes2);
    AFPS_CUDA(ctx, cudaStreamWaitEvent(stream, ctx->ev_done, 0));
    AFPS_CUDA(ctx, cudaMemcpyAsync(dst.p, ctx->stage[s].p, total, cudaMemcpyHostToDevice, stream));
    AFPS_CUDA(ctx, cudaEventRecord(ctx->stage_ev[s], stream));
    return AFPS_OK;
}

// The public batched layout: cloud b is points [pt_off[b], pt_off[b+1]),
// outputs [out_off[b], out_off[b+1]).
int build_plan_consecutive(afps_ctx* ctx, const int64_t* pt_off, int32_t B, const int32_t* C,
                           const int32_t* M, const int32_t* K, const int64_t* start,
                           const int64_t* out_off, BatchPlan& plan,
                           const uint32_t* method = nullptr, bool merge = true) {
    if (B < 1 || !pt_off || !out_off)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "batched call: B < 1 or a NULL host array");
    std::vector<int64_t> pb((size_t)B), np((size_t)B), ob((size_t)B), oc((size_t)B);
    for (int32_t b = 0; b < B; ++b) {
        pb[b] = pt_off[b];
        np[b] = pt_off[b + 1] - pt_off[b];
        ob[b] = out_off[b];
        oc[b] = out_off[b + 1] - out_off[b];
    }
    return build_plan(ctx, B, pb.data(), np.data(), ob.data(), oc.data(), C, M, K, start, plan,
                      method, merge);
}

// Run a plan out of the context's shared workspace (no graph).
int run_plan(afps_ctx* ctx, const BatchPlan& plan, const float* d_xyz, int32_t* d_out,
             cudaStream_t stream, bool host_resident = false) {
    const size_t bytes = plan.items.size() * sizeof(ItemDesc);  // a multiple of 16
    const size_t cbytes = plan.clouds.size() * sizeof(afps::CloudRec);
    bool table = cbytes > 0;  // some class reads the item table or cloud records
    bool queue = false;       // some class uses a work-queue counter
    for (const ClassPlan& cp : plan.classes) {
        table = table || !cp.uniform;
        queue = queue || uses_queue(cp.v, cp.count);
    }
    if (queue) {  // a new counter buffer is cleared after the workspace's last use
        AFPS_CUDA(ctx, cudaStreamWaitEvent(stream, ctx->ev_done, 0));
        int grc = grow_counters(ctx, ctx->counters, plan.classes.size(), stream);
        if (grc != AFPS_OK) return grc;
    }
    if (table) {  // the upload waits for the workspace's last use
        int urc = upload(ctx, ctx->items, plan.items.data(), bytes, stream, plan.clouds.data(),
                         cbytes);
        if (urc != AFPS_OK) return urc;
    }
    const ItemDesc* d_items = static_cast<const ItemDesc*>(ctx->items.p);
    const afps::CloudRec* d_clouds = reinterpret_cast<const afps::CloudRec*>(
        static_cast<const char*>(ctx->items.p) + bytes);
    unsigned int* counters = static_cast<unsigned int*>(ctx->counters.p);
    for (size_t i = 0; i < plan.classes.size(); ++i) {
        const ClassPlan& cp = plan.classes[i];
        afps::SingleCloud sc = cp.single;
        if (cp.cloud_first >= 0) sc.clouds = d_clouds + cp.cloud_first;
        int rc = launch_class(ctx, cp.v, cp.npdu, cp.uniform ? nullptr : d_items + cp.first,
                              cp.count, counters + i, d_xyz, d_out, stream, host_resident,
                              cp.uniform ? &sc : nullptr);
        if (rc != AFPS_OK) return rc;
    }
    // the workspace's last use, for ordering its next upload (none used: no record)
    if (table || queue) AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, stream));
    return AFPS_OK;
}

std::string graph_key(const float* d_xyz, int32_t* d_out, const int64_t* pt_off, int32_t B,
                      const int32_t* C, const int32_t* M, const int32_t* K,
                      const int64_t* start, const int64_t* out_off,
                      const uint32_t* method = nullptr) {
    std::string k;
    k.reserve(64 + (size_t)B * 40);
    auto put = [&](const void* p, size_t n) { k.append(static_cast<const char*>(p), n); };
    put(&d_xyz, sizeof d_xyz);
    put(&d_out, sizeof d_out);
    put(&B, sizeof B);
    put(pt_off, sizeof(int64_t) * (B + 1));
    put(out_off, sizeof(int64_t) * (B + 1));
    put(C, sizeof(int32_t) * B);
    put(M, sizeof(int32_t) * B);
    put(K, sizeof(int32_t) * B);
    put(start, sizeof(int64_t) * B);
    if (method) put(method, sizeof(uint32_t) * B);
    return k;
}

void drop_graph(GraphEntry& g) {
    if (g.exec) cudaGraphExecDestroy(g.exec);
    g.exec = nullptr;
    g.items.release();
    g.counters.release();
    g.xyz.release();
    g.out.release();
}

void clear_graphs(afps_ctx* ctx) {
    if (ctx->graphs.empty()) return;
    cudaDeviceSynchronize();
    for (auto& kv : ctx->graphs) drop_graph(kv.second);
    ctx->graphs.clear();
}

// Capture the plan's launches (counter resets + one kernel per class) into a
// graph that owns its own item table, so replays need no upload.
int make_graph(afps_ctx* ctx, const BatchPlan& plan, const float* d_xyz, int32_t* d_out,
               GraphEntry& g, const float* h_xyz = nullptr, size_t xyz_bytes = 0,
               int32_t* h_out = nullptr, size_t out_bytes = 0, bool host_resident = false) {
    const size_t bytes = plan.items.size() * sizeof(ItemDesc);
    AFPS_CUDA(ctx, grow(ctx, g.items, bytes));
    AFPS_CUDA(ctx, grow(ctx, g.counters, plan.classes.size() * sizeof(unsigned int)));
    // the graph's own queue counters start at zero; each replay leaves them so
    AFPS_CUDA(ctx, cudaMemset(g.counters.p, 0, g.counters.bytes));
    if (bytes)  // classes of equal-cloud runs need no table
        AFPS_CUDA(ctx, cudaMemcpy(g.items.p, plan.items.data(), bytes, cudaMemcpyHostToDevice));
    const ItemDesc* d_items = static_cast<const ItemDesc*>(g.items.p);
    unsigned int* counters = static_cast<unsigned int*>(g.counters.p);
    AFPS_CUDA(ctx, cudaStreamBeginCapture(ctx->capture, cudaStreamCaptureModeThreadLocal));
    const int64_t before = ctx->launches;
    int rc = AFPS_OK;
    if (h_xyz && cudaMemcpyAsync(const_cast<float*>(d_xyz), h_xyz, xyz_bytes,
                                 cudaMemcpyHostToDevice, ctx->capture) != cudaSuccess)
        rc = AFPS_ERR_CUDA;
    for (size_t i = 0; i < plan.classes.size() && rc == AFPS_OK; ++i) {
        const ClassPlan& cp = plan.classes[i];
        rc = launch_class(ctx, cp.v, cp.npdu, d_items + cp.first, cp.count, counters + i, d_xyz,
                          d_out, ctx->capture, host_resident, cp.run());
    }
    if (rc == AFPS_OK && h_out &&
        cudaMemcpyAsync(h_out, d_out, out_bytes, cudaMemcpyDeviceToHost, ctx->capture) !=
            cudaSuccess)
        rc = AFPS_ERR_CUDA;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamEndCapture(ctx->capture, &graph);
    g.kernels = ctx->launches - before;
    ctx->launches = before;  // capture launched nothing yet
    if (rc != AFPS_OK) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaGraphInstantiate");
    return AFPS_OK;
}

// AFPS_FLAG_AUTOTUNE: the first call with an argument set any of whose shape
// classes has no tuned variant yet runs the autotuner on it (synchronously;
// the call then samples as usual).
int tune_if_new(afps_ctx* ctx, const float* d_xyz, const int64_t* pt_off, int32_t B,
                const int32_t* C, const int32_t* M, const int32_t* K, const int64_t* start,
                const int64_t* out_off, int32_t* d_out, cudaStream_t stream,
                const uint32_t* method) {
    const std::string key = graph_key(nullptr, nullptr, pt_off, B, C, M, K, start, out_off, method);
    if (ctx->checked.count(key)) return AFPS_OK;
    BatchPlan plan;  // the classes the tuner times (unmerged)
    int rc = build_plan_consecutive(ctx, pt_off, B, C, M, K, start, out_off, plan, method, false);
    if (rc != AFPS_OK) return rc;
    bool tuned = true;
    for (const ClassPlan& cp : plan.classes)
        tuned = tuned && ctx->tuned.count(class_key(cp.npdu, cp.n_max, cp.c_max, cp.count)) > 0;
    if (!tuned) {
        rc = afps_autotune_batched(ctx, d_xyz, pt_off, B, C, M, K, start, out_off, d_out, stream);
        if (rc < 0) return rc;
    }
    if (ctx->checked.size() >= kMaxPlans) ctx->checked.clear();
    ctx->checked.insert(key);
    return AFPS_OK;
}

int batched_device(afps_ctx* ctx, const float* d_xyz, const int64_t* pt_off, int32_t B,
                   const int32_t* C, const int32_t* M, const int32_t* K, const int64_t* start,
                   const int64_t* out_off, int32_t* d_out, cudaStream_t stream,
                   const uint32_t* method = nullptr, bool host_resident = false) {
    if (!d_xyz || !d_out) return fail(ctx, AFPS_ERR_INVALID_ARG, "batched call: NULL device pointer");
    if (reinterpret_cast<uintptr_t>(d_xyz) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "batched call: xyz and out must be 4-byte aligned");
    if (B < 1 || !pt_off || !C || !M || !K || !start || !out_off)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "batched call: B < 1 or a NULL host array");
    if ((ctx->flags & AFPS_FLAG_AUTOTUNE) && !host_resident) {  // the tuner stages by bulk copy
        int rc = tune_if_new(ctx, d_xyz, pt_off, B, C, M, K, start, out_off, d_out, stream, method);
        if (rc != AFPS_OK) return rc;
    }
    if (!(ctx->flags & AFPS_FLAG_GRAPH) || host_resident) {
        // plans depend on the host arrays (and the tuning) only, not on the
        // device pointers: a repeated argument set skips validation and planning
        const std::string key =
            graph_key(nullptr, nullptr, pt_off, B, C, M, K, start, out_off, method);
        auto it = ctx->plans.find(key);
        if (it == ctx->plans.end()) {
            BatchPlan plan;
            int rc = build_plan_consecutive(ctx, pt_off, B, C, M, K, start, out_off, plan, method);
            if (rc != AFPS_OK) return rc;
            if (ctx->plans.size() >= kMaxPlans) ctx->plans.clear();
            it = ctx->plans.emplace(key, std::move(plan)).first;
        }
        return run_plan(ctx, it->second, d_xyz, d_out, stream, host_resident);
    }
    const std::string key = graph_key(d_xyz, d_out, pt_off, B, C, M, K, start, out_off, method);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        BatchPlan plan;
        int rc = build_plan_consecutive(ctx, pt_off, B, C, M, K, start, out_off, plan, method);
        if (rc != AFPS_OK) return rc;
        if (ctx->graphs.size() >= kMaxGraphs) {  // evict the least recently used
            auto victim = ctx->graphs.begin();
            for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
                if (j->second.last_use < victim->second.last_use) victim = j;
            cudaDeviceSynchronize();
            drop_graph(victim->second);
            ctx->graphs.erase(victim);
        }
        GraphEntry g;
        rc = make_graph(ctx, plan, d_xyz, d_out, g);
        if (rc != AFPS_OK) {
            drop_graph(g);
            return rc;
        }
        it = ctx->graphs.emplace(key, g).first;
    }
    it->second.last_use = ++ctx->tick;
    AFPS_CUDA(ctx, cudaGraphLaunch(it->second.exec, stream));
    ctx->launches += it->second.kernels;
    return AFPS_OK;
}

// Tuning cache: one line per class, "key kind P W CS occ [skip]".
// Page-locked host memory: true, with *dev its device address when it is
// mapped into the device's address space (else nullptr).  One driver query.
bool pinned_address(const void* p, void** dev) {
    *dev = nullptr;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (at.type != cudaMemoryTypeHost) return false;
    *dev = at.devicePointer;
    return true;
}

// afps_sample_batched_host with pinned buffers and AFPS_FLAG_GRAPH: one graph
// per argument set.  When both buffers are mapped into the device's address
// space (page-locked host memory; on Grace-Blackwell the GPU reaches it over
// the coherent C2C link) the kernels read the points and write the indices
// in host memory directly, with plain loads and stores; otherwise the graph
// holds the host->device copy, the sampling launches and the device->host
// copy around its own device staging.  A call is one replay and a wait.
int host_graph_call(afps_ctx* ctx, const float* h_xyz, const int64_t* pt_off, int32_t B,
                    const int32_t* C, const int32_t* M, const int32_t* K, const int64_t* start,
                    const int64_t* out_off, int32_t* h_out, size_t xyz_bytes, size_t out_bytes,
                    cudaStream_t stream, bool sync) {
    std::string key = "H" + graph_key(h_xyz, h_out, pt_off, B, C, M, K, start, out_off);
    auto it = ctx->graphs.find(key);
    if (it == ctx->graphs.end()) {
        BatchPlan plan;
        int rc = build_plan_consecutive(ctx, pt_off, B, C, M, K, start, out_off, plan);
        if (rc != AFPS_OK) return rc;
        if (ctx->graphs.size() >= kMaxGraphs) {
            auto victim = ctx->graphs.begin();
            for (auto j = ctx->graphs.begin(); j != ctx->graphs.end(); ++j)
                if (j->second.last_use < victim->second.last_use) victim = j;
            cudaDeviceSynchronize();
            drop_graph(victim->second);
            ctx->graphs.erase(victim);
        }
        GraphEntry g;
        void* dx = nullptr;
        void* dout = nullptr;
        const bool mapped =
            cudaHostGetDevicePointer(&dx, const_cast<float*>(h_xyz), 0) == cudaSuccess &&
            cudaHostGetDevicePointer(&dout, h_out, 0) == cudaSuccess && dx && dout &&
            reinterpret_cast<uintptr_t>(dx) % 4 == 0 && reinterpret_cast<uintptr_t>(dout) % 4 == 0;
        cudaGetLastError();
        if (mapped) {
            rc = make_graph(ctx, plan, static_cast<const float*>(dx), static_cast<int32_t*>(dout),
                            g, nullptr, 0, nullptr, 0, true);
        } else {
            if (grow(ctx, g.xyz, xyz_bytes) != cudaSuccess || grow(ctx, g.out, out_bytes) != cudaSuccess) {
                cudaGetLastError();
                drop_graph(g);
                return fail(ctx, AFPS_ERR_NO_MEMORY, "afps_sample_batched_host: device staging");
            }
            rc = make_graph(ctx, plan, static_cast<const float*>(g.xyz.p),
                            static_cast<int32_t*>(g.out.p), g, h_xyz, xyz_bytes, h_out, out_bytes);
        }
        if (rc != AFPS_OK) {
            drop_graph(g);
            return rc;
        }
        it = ctx->graphs.emplace(key, g).first;
    }
    it->second.last_use = ++ctx->tick;
    AFPS_CUDA(ctx, cudaGraphLaunch(it->second.exec, stream));
    ctx->launches += it->second.kernels;
    if (sync) AFPS_CUDA(ctx, cudaStreamSynchronize(stream));
    return AFPS_OK;
}

// The device a tuning file belongs to: name, SM count and compute capability.
std::string device_signature(int device) {
    cudaDeviceProp prop{};
    if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) {
        cudaGetLastError();
        return "unknown";
    }
    std::ostringstream os;
    for (const char* c = prop.name; *c; ++c) os << (*c == ' ' ? '_' : *c);
    os << " sms=" << prop.multiProcessorCount << " cc=" << prop.major << '.' << prop.minor;
    return os.str();
}

// Tuning file: a "# device <signature>" line, then one line per class,
// "key kind P W CS occ skip".  A file written on another kind of device is
// ignored (its variants would be valid but not tuned for this one).
int load_tuning(afps_ctx* ctx, const std::string& path) {
    std::ifstream f(path);
    if (!f) return 0;
    std::string line;
    int n = 0;
    const std::string want = "# device " + device_signature(ctx->device);
    while (std::getline(f, line)) {
        if (line.rfind("# device ", 0) == 0) {
            if (line != want) return 0;
            continue;
        }
        std::istringstream is(line);
        std::string key;
        Variant v{};
        if (!(is >> key >> v.kind >> v.P >> v.W >> v.CS >> v.occ)) continue;
        if (!(is >> v.skip)) v.skip = 0;
        if (afps::variant_supported(v)) {
            ctx->tuned[key] = v;
            ++n;
        }
    }
    return n;
}

}  // namespace

// ============================================================ internal API
namespace afps {

int gather_run(afps_ctx* ctx, const GatherDesc* descs, int32_t B, const float* in_xyz,
               const int32_t* in_frame, const int32_t* sel, float* out_xyz, int32_t* out_frame,
               int32_t* sel_frame, cudaStream_t stream) {
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    int32_t max_n = 1;
    for (int32_t b = 0; b < B; ++b) {
        const GatherDesc& g = descs[b];
        if (g.n < 1 || g.n > kGatherMaxPoints || g.c < 0 || g.c >= 65536 || g.in_xyz < 0 ||
            g.sel < 0 || g.out_xyz < 0 || (g.in_frame >= 0 && !in_frame) ||
            (g.out_frame >= 0 && !out_frame) || (g.sel_frame >= 0 && !sel_frame)) {
            std::ostringstream os;
            os << "gather: cloud " << b << " has " << g.n << " points and " << g.c
               << " samples (need 1 <= n <= " << kGatherMaxPoints
               << ", 0 <= c < 65536) or a frame offset without its array";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        max_n = std::max(max_n, g.n);
    }
    int rc = upload(ctx, ctx->items, descs, (size_t)B * sizeof(GatherDesc), stream);
    if (rc != AFPS_OK) return rc;
    cudaError_t e = launch_gather(static_cast<const GatherDesc*>(ctx->items.p), B, max_n, in_xyz,
                                  in_frame, sel, out_xyz, out_frame, sel_frame, stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather launch");
    ctx->launches += 1;
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, stream));
    return AFPS_OK;
}

// Reserve the shared workspace (device item table and every slot of the
// pinned upload ring) for tables of up to `bytes`, so that a runtime whose
// tables grow over time (the server) does not reallocate them mid-stream.
int reserve_workspace(afps_ctx* ctx, size_t bytes) {
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    AFPS_CUDA(ctx, cudaDeviceSynchronize());  // nothing may still read the old buffers
    AFPS_CUDA(ctx, grow(ctx, ctx->items, bytes));
    for (int s = 0; s < kStageSlots; ++s) AFPS_CUDA(ctx, grow(ctx, ctx->stage[s], bytes));
    return AFPS_OK;
}

int clone_context(afps_ctx* src, afps_ctx** out) {
    if (!src || !out) return AFPS_ERR_INVALID_ARG;
    *out = nullptr;
    afps_config cfg{};
    cfg.device = src->device;
    cfg.flags = src->flags;
    cfg.timeout_ns = (int64_t)src->timeout_ns;
    afps_ctx* c = nullptr;
    const int rc = afps_create(&c, &cfg);
    if (rc != AFPS_OK) return rc;
    {
        DeviceGuard guard(c->device);
        cudaFree(c->d_status);
        cudaGetLastError();
    }
    c->d_status = src->d_status;
    c->status_borrowed = true;
    c->tuned = src->tuned;
    *out = c;
    return AFPS_OK;
}

void copy_error(afps_ctx* to, const afps_ctx* from) {
    if (to && from && to != from) to->last_error = from->last_error;
}

int sample_scattered(afps_ctx* ctx, const float* xyz, int32_t B, const int64_t* pt_begin,
                     const int64_t* n_pts, const int32_t* C, const int32_t* M, const int32_t* K,
                     const int64_t* start, int32_t* out, const int64_t* out_begin,
                     cudaStream_t stream) {
    if (!ctx || !xyz || !out) return AFPS_ERR_INVALID_ARG;
    std::vector<int64_t> cap((size_t)std::max(B, 1));
    for (int32_t b = 0; b < B; ++b) cap[b] = C[b];
    BatchPlan plan;
    int rc = build_plan(ctx, B, pt_begin, n_pts, out_begin, cap.data(), C, M, K, start, plan,
                        nullptr, true, true);
    if (rc != AFPS_OK) return rc;
    return run_plan(ctx, plan, xyz, out, stream);
}

}  // namespace afps

// ====================================================================== ABI
extern "C" {

int afps_create(afps_ctx** out, const afps_config* cfg) {
    if (!out) return AFPS_ERR_INVALID_ARG;
    *out = nullptr;
    afps_ctx* ctx = new (std::nothrow) afps_ctx();
    if (!ctx) return AFPS_ERR_NO_MEMORY;
    if (cfg) {
        ctx->device = cfg->device;
        ctx->flags = cfg->flags;
        if (cfg->timeout_ns > 0) ctx->timeout_ns = (uint64_t)cfg->timeout_ns;
        if (cfg->tune_cache) ctx->tune_path = cfg->tune_cache;
    }
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ctx->device < 0 || ctx->device >= ndev) {
        cudaGetLastError();
        delete ctx;
        return AFPS_ERR_CUDA;
    }
    DeviceGuard guard(ctx->device);
    cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount,
                                           ctx->device);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->ev_done, cudaEventDisableTiming);
    for (int i = 0; i < kStageSlots && e == cudaSuccess; ++i)
        e = cudaEventCreateWithFlags(&ctx->stage_ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->capture, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventRecord(ctx->ev_done, ctx->capture);
    for (int i = 0; i < kStageSlots && e == cudaSuccess; ++i)
        e = cudaEventRecord(ctx->stage_ev[i], ctx->capture);
    if (e != cudaSuccess) {
        cudaGetLastError();
        afps_destroy(ctx);
        return AFPS_ERR_CUDA;
    }
    if (!ctx->tune_path.empty()) load_tuning(ctx, ctx->tune_path);
    *out = ctx;
    return AFPS_OK;
}

void afps_destroy(afps_ctx* ctx) {
    if (!ctx) return;
    {
        DeviceGuard guard(ctx->device);
        cudaDeviceSynchronize();
        for (auto& kv : ctx->graphs) drop_graph(kv.second);
        ctx->graphs.clear();
        ctx->items.release();
        ctx->counters.release();
        ctx->xyz_stage.release();
        ctx->out_stage.release();
        ctx->sort_scratch.release();
        ctx->cov_scratch.release();
        for (int i = 0; i < kStageSlots; ++i) {
            ctx->stage[i].release();
            if (ctx->stage_ev[i]) cudaEventDestroy(ctx->stage_ev[i]);
        }
        if (ctx->d_status && !ctx->status_borrowed) cudaFree(ctx->d_status);
        if (ctx->ev_done) cudaEventDestroy(ctx->ev_done);
        if (ctx->capture) cudaStreamDestroy(ctx->capture);
        cudaGetLastError();
    }
    delete ctx;
}

int afps_sample(afps_ctx* ctx, const float* d_xyz, int64_t N, int32_t C, int32_t M,
                int32_t npdu_window, int64_t start_idx, int32_t* d_out, void* stream) {
    AFPS_TRACE("afps_sample");
    return afps_sample_ex(ctx, d_xyz, N, C, M, npdu_window, start_idx, 0u, d_out, stream);
}

int afps_sample_ex(afps_ctx* ctx, const float* d_xyz, int64_t N, int32_t C, int32_t M,
                   int32_t npdu_window, int64_t start_idx, uint32_t method, int32_t* d_out,
                   void* stream) {
    AFPS_TRACE("afps_sample_ex");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (method > AFPS_METHOD_ALL)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_sample_ex: unknown method bits");
    if (!d_xyz || !d_out)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_sample: NULL device pointer");
    if (reinterpret_cast<uintptr_t>(d_xyz) % 4 || reinterpret_cast<uintptr_t>(d_out) % 4)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_sample: xyz and out must be 4-byte aligned");
    CloudCheck chk = check_cloud(N, C, M, npdu_window, start_idx);
    if (chk.code != AFPS_OK) return fail(ctx, chk.code, "afps_sample: " + chk.msg);
    DeviceGuard guard(ctx->device);
    const bool npdu = npdu_window > 0;
    ItemDesc wsides{};
    window_sides(npdu_window, method, wsides);
    const bool narrow = wsides.kl + wsides.kr <= 16 && !(wsides.flags & afps::ITEM_FULL_FIRST);
    const Variant v = choose_variant(ctx, npdu, chk.n_max, chk.c_max, (size_t)M, narrow);
    LaunchArgs a{};
    a.xyz = d_xyz;
    a.items = nullptr;
    a.single.pt_off = 0;
    a.single.out_off = 0;
    a.single.N = (int32_t)N;
    a.single.C = C;
    a.single.M = M;
    {
        ItemDesc w{};
        window_sides(npdu_window, method, w);
        a.single.kl = w.kl;
        a.single.kr = w.kr;
        a.single.flags = w.flags;
    }
    a.single.start_r = chk.start_r;
    a.single.wide = (int64_t)M * N > (int64_t)UINT32_MAX ? 1 : 0;
    a.single.m_magic = afps::div_magic(M);
    a.n_items = M;
    a.out = d_out;
    a.counter = nullptr;
    a.status = ctx->d_status;
    a.timeout_ns = ctx->timeout_ns;
    a.stall = stall_bits(ctx->flags);
    a.npdu_skip = v.skip ? 1u : 0u;
    cudaError_t e = afps::launch_sector(v, npdu, a, grid_for(v, (size_t)M),
                                        static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "afps_sample launch");
    ctx->launches += 1;
    return AFPS_OK;
}

int afps_sample_batched(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off, int32_t B,
                        const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
                        const int64_t* h_start, const int64_t* h_out_off, int32_t* d_out,
                        void* stream) {
    AFPS_TRACE("afps_sample_batched");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    return batched_device(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, d_out,
                          static_cast<cudaStream_t>(stream));
}

int afps_sample_batched_ex(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off,
                           int32_t B, const int32_t* h_C, const int32_t* h_M,
                           const int32_t* h_win, const int64_t* h_start,
                           const uint32_t* h_method, const int64_t* h_out_off, int32_t* d_out,
                           void* stream) {
    AFPS_TRACE("afps_sample_batched_ex");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (!h_method) return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_sample_batched_ex: NULL h_method");
    DeviceGuard guard(ctx->device);
    return batched_device(ctx, d_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, d_out,
                          static_cast<cudaStream_t>(stream), h_method);
}

}  // extern "C"

namespace {

// afps_sample_batched_host(_async).  Page-locked buffers: a cached graph
// (AFPS_FLAG_GRAPH) or, when the buffers are mapped, direct launches whose
// kernels read the points and write the indices in host memory; otherwise
// copies through context-owned device staging (pageable memory: sync only).
int host_call(afps_ctx* ctx, const float* h_xyz, const int64_t* h_pt_off, int32_t B,
              const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
              const int64_t* h_start, const int64_t* h_out_off, int32_t* h_out, void* stream,
              bool sync, const char* name) {
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (!h_xyz || !h_out || !h_pt_off || !h_out_off || B < 1)
        return fail(ctx, AFPS_ERR_INVALID_ARG, std::string(name) + ": NULL argument or B < 1");
    if (h_pt_off[0] != 0 || h_out_off[0] != 0)
        return fail(ctx, AFPS_ERR_INVALID_ARG,
                    std::string(name) + ": h_pt_off[0] and h_out_off[0] must be 0");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    const size_t xyz_bytes = (size_t)h_pt_off[B] * 3 * sizeof(float);
    const size_t out_bytes = (size_t)h_out_off[B] * sizeof(int32_t);
    void* dx = nullptr;
    void* dout = nullptr;
    const bool pinned = pinned_address(h_xyz, &dx) && pinned_address(h_out, &dout);
    if (!sync && !pinned)
        return fail(ctx, AFPS_ERR_INVALID_ARG, std::string(name) + ": needs page-locked buffers");
    if ((ctx->flags & AFPS_FLAG_GRAPH) && pinned)
        return host_graph_call(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off,
                               h_out, xyz_bytes, out_bytes, st, sync);
    if (pinned) {
        if (dx && dout) {  // mapped: the kernels work in host memory
            int rc = batched_device(ctx, static_cast<const float*>(dx), h_pt_off, B, h_C, h_M,
                                    h_win, h_start, h_out_off, static_cast<int32_t*>(dout), st,
                                    nullptr, true);
            if (rc != AFPS_OK) return rc;
            if (sync) AFPS_CUDA(ctx, cudaStreamSynchronize(st));
            return AFPS_OK;
        }
    }
    AFPS_CUDA(ctx, grow(ctx, ctx->xyz_stage, xyz_bytes));
    AFPS_CUDA(ctx, grow(ctx, ctx->out_stage, out_bytes));
    AFPS_CUDA(ctx, cudaStreamWaitEvent(st, ctx->ev_done, 0));
    AFPS_CUDA(ctx, cudaMemcpyAsync(ctx->xyz_stage.p, h_xyz, xyz_bytes, cudaMemcpyHostToDevice, st));
    int rc = batched_device(ctx, static_cast<const float*>(ctx->xyz_stage.p), h_pt_off, B, h_C,
                            h_M, h_win, h_start, h_out_off,
                            static_cast<int32_t*>(ctx->out_stage.p), st);
    if (rc != AFPS_OK) {
        cudaStreamSynchronize(st);
        return rc;
    }
    AFPS_CUDA(ctx, cudaMemcpyAsync(h_out, ctx->out_stage.p, out_bytes, cudaMemcpyDeviceToHost, st));
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, st));
    if (sync) AFPS_CUDA(ctx, cudaStreamSynchronize(st));
    return AFPS_OK;
}

}  // namespace

extern "C" {

int afps_sample_batched_host(afps_ctx* ctx, const float* h_xyz, const int64_t* h_pt_off,
                             int32_t B, const int32_t* h_C, const int32_t* h_M,
                             const int32_t* h_win, const int64_t* h_start,
                             const int64_t* h_out_off, int32_t* h_out, void* stream) {
    AFPS_TRACE("afps_sample_batched_host");
    return host_call(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, h_out, stream,
                     true, "afps_sample_batched_host");
}

int afps_sample_batched_host_async(afps_ctx* ctx, const float* h_xyz, const int64_t* h_pt_off,
                                   int32_t B, const int32_t* h_C, const int32_t* h_M,
                                   const int32_t* h_win, const int64_t* h_start,
                                   const int64_t* h_out_off, int32_t* h_out, void* stream) {
    AFPS_TRACE("afps_sample_batched_host_async");
    return host_call(ctx, h_xyz, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, h_out, stream,
                     false, "afps_sample_batched_host_async");
}

int afps_gather_levels(afps_ctx* ctx, int32_t B, const int64_t* h_in_pt_off,
                       const float* d_in_xyz, const int32_t* d_in_frame,
                       const int64_t* h_sel_off, const int32_t* d_sel, float* d_out_xyz,
                       int32_t* d_out_frame, int32_t* d_sel_frame, void* stream) {
    AFPS_TRACE("afps_gather_levels");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (B < 1 || !h_in_pt_off || !h_sel_off || !d_in_xyz || !d_sel || !d_out_xyz)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_gather_levels: NULL argument or B < 1");
    std::vector<afps::GatherDesc> descs((size_t)B);
    for (int32_t b = 0; b < B; ++b) {
        const int64_t n = h_in_pt_off[b + 1] - h_in_pt_off[b];
        const int64_t c = h_sel_off[b + 1] - h_sel_off[b];
        afps::GatherDesc& g = descs[b];
        g.in_xyz = h_in_pt_off[b];
        g.in_frame = d_in_frame ? h_in_pt_off[b] : -1;
        g.sel = h_sel_off[b];
        g.out_xyz = h_sel_off[b];
        g.out_frame = d_out_frame ? h_sel_off[b] : -1;
        g.sel_frame = d_sel_frame ? h_sel_off[b] : -1;
        g.n = (int32_t)std::min<int64_t>(n, INT32_MAX);
        g.c = (int32_t)std::min<int64_t>(c, INT32_MAX);
        if (n < 1 || c < 0) g.n = -1;  // rejected below
    }
    DeviceGuard guard(ctx->device);
    return afps::gather_run(ctx, descs.data(), B, d_in_xyz, d_in_frame, d_sel, d_out_xyz,
                            d_out_frame, d_sel_frame, static_cast<cudaStream_t>(stream));
}

int afps_sort_by_key(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                     int32_t key, float* d_xyz_sorted, int32_t* d_perm, void* stream) {
    AFPS_TRACE("afps_sort_by_key");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (B < 1 || !h_pt_off || !d_xyz || !d_xyz_sorted || !d_perm || key < AFPS_KEY_X ||
        key > AFPS_KEY_AZIMUTH || h_pt_off[0] < 0)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_sort_by_key: bad argument");
    // small clouds: one CTA each (global scratch); large ones: one cluster
    // each, held in distributed shared memory
    std::vector<afps::SortDesc> small, large;
    int64_t small_points = 0;
    int32_t large_max = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t n = h_pt_off[b + 1] - h_pt_off[b];
        if (n < 0 || n > INT32_MAX) {
            std::ostringstream os;
            os << "afps_sort_by_key: cloud " << b << " has " << n << " points";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        const afps::SortDesc sd{h_pt_off[b], (int32_t)n, 0};
        if (n > afps::kSortClusterMin && n <= afps::sort_cluster_capacity()) {
            large.push_back(sd);
            large_max = std::max(large_max, (int32_t)n);
        } else {
            small.push_back(sd);
            small_points = std::max(small_points, h_pt_off[b + 1]);
        }
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // scratch of the small clouds' sort: keys and indices, twice (ping-pong),
    // indexed by point; earlier users are ordered before a reallocation by
    // cudaFree's device synchronisation
    if (!small.empty()) AFPS_CUDA(ctx, grow(ctx, ctx->sort_scratch, (size_t)small_points * 16 + 16));
    std::vector<afps::SortDesc> descs(small);
    descs.insert(descs.end(), large.begin(), large.end());
    int rc = upload(ctx, ctx->items, descs.data(), descs.size() * sizeof(afps::SortDesc), st);
    if (rc != AFPS_OK) return rc;
    const afps::SortDesc* d_descs = static_cast<const afps::SortDesc*>(ctx->items.p);
    if (!small.empty()) {
        const int64_t total = small_points;
        unsigned char* base = static_cast<unsigned char*>(ctx->sort_scratch.p);
        uint32_t* keys_a = reinterpret_cast<uint32_t*>(base);
        int32_t* idx_a = reinterpret_cast<int32_t*>(base + 4 * total);
        uint32_t* keys_b = reinterpret_cast<uint32_t*>(base + 8 * total);
        int32_t* idx_b = reinterpret_cast<int32_t*>(base + 12 * total);
        cudaError_t e = afps::launch_sort(d_descs, (int32_t)small.size(), d_xyz, key, keys_a,
                                          idx_a, keys_b, idx_b, d_xyz_sorted, d_perm, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "sort launch");
        ctx->launches += 1;
    }
    if (!large.empty()) {
        cudaError_t e = afps::launch_sort_cluster(d_descs + small.size(), (int32_t)large.size(),
                                                  large_max, d_xyz, key, d_xyz_sorted, d_perm, st);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cluster sort launch");
        ctx->launches += 1;
    }
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, st));
    return AFPS_OK;
}

int afps_coverage_radius(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                         const int64_t* h_sel_off, const int32_t* d_sel, double* d_radius,
                         void* stream) {
    AFPS_TRACE("afps_coverage_radius");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (B < 1 || B > 65535 || !h_pt_off || !h_sel_off || !d_xyz || !d_sel || !d_radius)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_coverage_radius: bad argument (1 <= B <= 65535)");
    std::vector<afps::CoverageDesc> descs((size_t)B);
    int32_t max_n = 1;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t n = h_pt_off[b + 1] - h_pt_off[b];
        const int64_t c = h_sel_off[b + 1] - h_sel_off[b];
        if (n < 1 || n > INT32_MAX || c < 1 || c > INT32_MAX || h_pt_off[b] < 0 ||
            h_sel_off[b] < 0) {
            std::ostringstream os;
            os << "afps_coverage_radius: cloud " << b << " has " << n << " points and " << c
               << " samples (need both >= 1)";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        descs[b] = afps::CoverageDesc{h_pt_off[b], h_sel_off[b], (int32_t)n, (int32_t)c};
        max_n = std::max<int32_t>(max_n, (int32_t)n);
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    AFPS_CUDA(ctx, grow(ctx, ctx->cov_scratch, sizeof(unsigned long long) * (size_t)B));
    int rc = upload(ctx, ctx->items, descs.data(), descs.size() * sizeof(afps::CoverageDesc), st);
    if (rc != AFPS_OK) return rc;
    cudaError_t e = afps::launch_coverage(
        static_cast<const afps::CoverageDesc*>(ctx->items.p), B, max_n, d_xyz, d_sel,
        static_cast<unsigned long long*>(ctx->cov_scratch.p), d_radius, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "coverage launch");
    ctx->launches += 2;
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, st));
    return AFPS_OK;
}

int afps_ball_query(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
                    const int64_t* h_sel_off, const int32_t* d_sel, float radius, int32_t K,
                    int32_t sorted_axis, int32_t* d_group, void* stream) {
    AFPS_TRACE("afps_ball_query");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (B < 1 || B > 65535 || !h_pt_off || !h_sel_off || !d_xyz || !d_sel || !d_group ||
        !(radius > 0.f) || K < 1 || sorted_axis < -1 || sorted_axis > 2)
        return fail(ctx, AFPS_ERR_INVALID_ARG,
                    "afps_ball_query: bad argument (1 <= B <= 65535, radius > 0, K >= 1, "
                    "sorted_axis in -1..2)");
    std::vector<afps::GroupDesc> descs((size_t)B);
    int32_t max_c = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t n = h_pt_off[b + 1] - h_pt_off[b];
        const int64_t c = h_sel_off[b + 1] - h_sel_off[b];
        if (n < 1 || n > INT32_MAX || c < 0 || c > INT32_MAX || h_pt_off[b] < 0 ||
            h_sel_off[b] < 0) {
            std::ostringstream os;
            os << "afps_ball_query: cloud " << b << " has " << n << " points and " << c
               << " centroids";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        descs[b] = afps::GroupDesc{h_pt_off[b], h_sel_off[b], (int32_t)n, (int32_t)c};
        max_c = std::max<int32_t>(max_c, (int32_t)c);
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload(ctx, ctx->items, descs.data(), descs.size() * sizeof(afps::GroupDesc), st);
    if (rc != AFPS_OK) return rc;
    cudaError_t e = afps::launch_ball_query(static_cast<const afps::GroupDesc*>(ctx->items.p), B,
                                            max_c, d_xyz, d_sel, radius, K, sorted_axis, d_group,
                                            st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "ball query launch");
    ctx->launches += 1;
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, st));
    return AFPS_OK;
}

int afps_knn(afps_ctx* ctx, int32_t B, const int64_t* h_pt_off, const float* d_xyz,
             const int64_t* h_sel_off, const int32_t* d_sel, int32_t K, int32_t sorted_axis,
             int32_t* d_group, float* d_dist2, void* stream) {
    AFPS_TRACE("afps_knn");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (B < 1 || B > 65535 || !h_pt_off || !h_sel_off || !d_xyz || !d_sel || !d_group || K < 1 ||
        K > 64 || sorted_axis < -1 || sorted_axis > 2)
        return fail(ctx, AFPS_ERR_INVALID_ARG,
                    "afps_knn: bad argument (1 <= B <= 65535, 1 <= K <= 64, sorted_axis in -1..2)");
    std::vector<afps::GroupDesc> descs((size_t)B);
    int32_t max_c = 0;
    for (int32_t b = 0; b < B; ++b) {
        const int64_t n = h_pt_off[b + 1] - h_pt_off[b];
        const int64_t c = h_sel_off[b + 1] - h_sel_off[b];
        if (n < K || n > INT32_MAX || c < 0 || c > INT32_MAX || h_pt_off[b] < 0 ||
            h_sel_off[b] < 0) {
            std::ostringstream os;
            os << "afps_knn: cloud " << b << " has " << n << " points (K = " << K << ") and "
               << c << " centroids";
            return fail(ctx, AFPS_ERR_INVALID_ARG, os.str());
        }
        descs[b] = afps::GroupDesc{h_pt_off[b], h_sel_off[b], (int32_t)n, (int32_t)c};
        max_c = std::max<int32_t>(max_c, (int32_t)c);
    }
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int rc = upload(ctx, ctx->items, descs.data(), descs.size() * sizeof(afps::GroupDesc), st);
    if (rc != AFPS_OK) return rc;
    cudaError_t e = afps::launch_knn(static_cast<const afps::GroupDesc*>(ctx->items.p), B, max_c,
                                     d_xyz, d_sel, K, sorted_axis, d_group, d_dist2, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "knn launch");
    if (max_c > 0) ctx->launches += 1;
    AFPS_CUDA(ctx, cudaEventRecord(ctx->ev_done, st));
    return AFPS_OK;
}

int afps_sync(afps_ctx* ctx, void* stream) {
    AFPS_TRACE("afps_sync");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    DeviceGuard guard(ctx->device);
    AFPS_CUDA(ctx, cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
    int status = 0;
    AFPS_CUDA(ctx, cudaMemcpy(&status, ctx->d_status, sizeof(int), cudaMemcpyDeviceToHost));
    if (status != 0) {
        AFPS_CUDA(ctx, cudaMemset(ctx->d_status, 0, sizeof(int)));
        if (status == afps::DEV_CHECK_FAILED)
            return fail(ctx, AFPS_ERR_DEVICE_CHECK,
                        "a device-side index check failed (debug build); the index was clamped");
        return fail(ctx, AFPS_ERR_TIMEOUT,
                    status == afps::DEV_TIMEOUT_STAGE
                        ? "a stage-in bulk copy did not complete within the timeout"
                    : status == afps::DEV_TIMEOUT_EXCHANGE
                        ? "a cluster record exchange did not complete within the timeout"
                        : "a bulk copy was still in flight after the drain timeout");
    }
    return AFPS_OK;
}

const char* afps_last_error(const afps_ctx* ctx) {
    return ctx ? ctx->last_error.c_str() : "NULL context";
}

int afps_autotune_batched(afps_ctx* ctx, const float* d_xyz, const int64_t* h_pt_off, int32_t B,
                          const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
                          const int64_t* h_start, const int64_t* h_out_off, int32_t* d_out,
                          void* stream) {
    AFPS_TRACE("afps_autotune_batched");
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (!d_xyz || !d_out) return fail(ctx, AFPS_ERR_INVALID_ARG, "autotune: NULL device pointer");
    DeviceGuard guard(ctx->device);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    BatchPlan plan;  // unmerged: every shape class is tuned on its own
    int rc = build_plan_consecutive(ctx, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, plan,
                                    nullptr, false);
    if (rc != AFPS_OK) return rc;
    // upload the table once, then time each candidate class by class
    rc = run_plan(ctx, plan, d_xyz, d_out, st);
    if (rc != AFPS_OK) return rc;
    cudaEvent_t e0, e1;
    AFPS_CUDA(ctx, cudaEventCreate(&e0));
    AFPS_CUDA(ctx, cudaEventCreate(&e1));
    // candidates may use a work queue where the plan's variants do not (one
    // more counter for the merged launches below)
    rc = grow_counters(ctx, ctx->counters, plan.classes.size() + 1, st);
    if (rc != AFPS_OK) return rc;
    const ItemDesc* d_items = static_cast<const ItemDesc*>(ctx->items.p);
    unsigned int* counters = static_cast<unsigned int*>(ctx->counters.p);
    // one warm-up round and three timed ones of four launches back to back
    // (a single launch of a small class lasts little longer than its launch
    // latency); < 0 if the variant cannot run
    auto time_launch = [&](const Variant& v, bool npdu, const ItemDesc* items, size_t count,
                           unsigned int* counter, const afps::SingleCloud* run) -> float {
        if (grid_for(v, count) < 1 || afps::max_active_clusters(v) < 1) return -1.f;
        float ms_sum = 0.f;
        bool ok = true;
        for (int rep = 0; rep < 4 && ok; ++rep) {
            if (cudaEventRecord(e0, st) != cudaSuccess) ok = false;
            for (int l = 0; l < 4 && ok; ++l)
                if (launch_class(ctx, v, npdu, items, count, counter, d_xyz, d_out, st, false,
                                 run) != AFPS_OK)
                    ok = false;
            if (ok && cudaEventRecord(e1, st) != cudaSuccess) ok = false;
            float ms = 0.f;
            if (ok && (cudaEventSynchronize(e1) != cudaSuccess ||
                       cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess))
                ok = false;
            if (rep > 0) ms_sum += ms;
        }
        if (!ok) {
            cudaGetLastError();
            return -1.f;
        }
        return ms_sum;
    };
    int tuned = 0;
    std::vector<float> best_of(plan.classes.size(), 0.f);
    for (size_t i = 0; i < plan.classes.size() && rc == AFPS_OK; ++i) {
        ClassPlan& cp = plan.classes[i];
        float best_ms = 1e30f;
        Variant best = cp.v;
        for (const Variant& v : candidate_variants(cp.n_max, cp.npdu, cp.narrow)) {
            const float ms = time_launch(v, cp.npdu, cp.uniform ? nullptr : d_items + cp.first,
                                         cp.count, counters + i, cp.run());
            if (ms >= 0.f && ms < best_ms) {
                best_ms = ms;
                best = v;
            }
        }
        ctx->tuned[class_key(cp.npdu, cp.n_max, cp.c_max, cp.count)] = best;
        cp.v = best;
        best_of[i] = best_ms;
        ++tuned;
    }
    // Consecutive NPDU table classes the window kernel can serve with one
    // template run as one launch when that is faster than their best
    // separate launches (one queue over all their items has a shorter tail);
    // their entries then name window variants with a common warp count,
    // which the planner merges (merge_window_classes).
    for (size_t i = 0; i < plan.classes.size();) {
        auto fits = [&](const ClassPlan& c) {
            return c.npdu && !c.uniform && c.n_max <= 32LL * afps::kWinMaxRows;
        };
        // (the pair kernel joins in when every class of the run is narrow)
        if (!fits(plan.classes[i])) {
            ++i;
            continue;
        }
        size_t j = i + 1;
        while (j < plan.classes.size() && fits(plan.classes[j]) &&
               plan.classes[j].first == plan.classes[j - 1].first + plan.classes[j - 1].count)
            ++j;
        if (j - i >= 2) {
            float separate = 0.f;
            size_t count = 0;
            int64_t n_max = 0;
            for (size_t c = i; c < j; ++c) {
                separate += best_of[c];
                count += plan.classes[c].count;
                n_max = std::max(n_max, plan.classes[c].n_max);
            }
            bool pairs_fit = afps::variant_supported(win2_variant(n_max));
            for (size_t c = i; c < j; ++c) pairs_fit = pairs_fit && plan.classes[c].narrow;
            float best_ms = separate;
            int best_w = 0, best_form = 0;  // form: 0 window, 1 window lean, 2 pairs
            for (int W : {1, 2, 4, 8})
                for (int form = 0; form < (pairs_fit ? 3 : 2); ++form) {
                    const Variant v = form == 2 ? win2_variant(n_max, W)
                                                : win_variant(n_max, W, form == 1);
                    if (!afps::variant_supported(v)) continue;
                    const float ms = time_launch(v, true, d_items + plan.classes[i].first, count,
                                                 counters + plan.classes.size(), nullptr);
                    if (ms >= 0.f && ms < best_ms) {
                        best_ms = ms;
                        best_w = W;
                        best_form = form;
                    }
                }
            for (size_t c = i; best_w && c < j; ++c) {
                ClassPlan& cp = plan.classes[c];
                cp.v = best_form == 2 ? win2_variant(cp.n_max, best_w)
                                      : win_variant(cp.n_max, best_w, best_form == 1);
                ctx->tuned[class_key(true, cp.n_max, cp.c_max, cp.count)] = cp.v;
            }
        }
        i = j;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    clear_graphs(ctx);  // graphs captured earlier may use other variants
    ctx->plans.clear();  // and so may cached plans
    ctx->last_error.clear();
    rc = run_plan(ctx, plan, d_xyz, d_out, st);
    return rc == AFPS_OK ? tuned : rc;
}

int afps_save_tuning(afps_ctx* ctx, const char* path) {
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    const std::string p = path ? std::string(path) : ctx->tune_path;
    if (p.empty()) return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_save_tuning: no path");
    std::ofstream f(p);
    if (!f) return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_save_tuning: cannot open " + p);
    f << "# device " << device_signature(ctx->device) << '\n';
    for (const auto& kv : ctx->tuned)
        f << kv.first << ' ' << kv.second.kind << ' ' << kv.second.P << ' ' << kv.second.W << ' '
          << kv.second.CS << ' ' << kv.second.occ << ' ' << kv.second.skip << '\n';
    return AFPS_OK;
}

int afps_describe_plan(afps_ctx* ctx, int64_t n_sector, int32_t c_sector, int32_t npdu_window,
                       int32_t n_items, char* buf, int32_t buf_len) {
    if (!ctx || !buf || buf_len < 1 || n_sector < 1 || n_sector > AFPS_MAX_SECTOR_POINTS ||
        n_items < 1)
        return AFPS_ERR_INVALID_ARG;
    const Variant v =
        choose_variant(ctx, npdu_window > 0, n_sector, c_sector, (size_t)n_items,
                       npdu_window <= 16);
    const std::string s = describe(v);
    snprintf(buf, (size_t)buf_len, "%s", s.c_str());
    return (int)s.size();
}

int afps_describe_batched(afps_ctx* ctx, const int64_t* h_pt_off, int32_t B,
                          const int32_t* h_C, const int32_t* h_M, const int32_t* h_win,
                          const int64_t* h_start, const int64_t* h_out_off, char* buf,
                          int32_t buf_len) {
    if (!ctx) return AFPS_ERR_INVALID_ARG;
    if (!buf || buf_len < 1 || B < 1 || !h_pt_off || !h_C || !h_M || !h_win || !h_start ||
        !h_out_off)
        return fail(ctx, AFPS_ERR_INVALID_ARG, "afps_describe_batched: NULL argument or B < 1");
    DeviceGuard guard(ctx->device);
    BatchPlan plan;
    int rc = build_plan_consecutive(ctx, h_pt_off, B, h_C, h_M, h_win, h_start, h_out_off, plan);
    if (rc != AFPS_OK) return rc;
    std::ostringstream os;
    for (size_t i = 0; i < plan.classes.size(); ++i)
        os << (i ? "; " : "") << describe(plan.classes[i].v) << " items=" << plan.classes[i].count;
    const std::string s = os.str();
    snprintf(buf, (size_t)buf_len, "%s", s.c_str());
    return (int)s.size();
}

int64_t afps_launch_count(const afps_ctx* ctx) { return ctx ? ctx->launches : 0; }

}  // extern "C"
