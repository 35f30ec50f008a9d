// afps_server.cu -- serving runtime: continuous batching of chained NPDU-AFPS
// requests over one device arena (see the afps_server_* block of afps.h).
//
// Each request owns one arena block laid out as
//   xyz (points, 12 B each):  frame N | cloud 1: C0 | ... | cloud L: C_{L-1}
//   int32:                    out_0: C0 | ... | out_{L-1} | frame index of
//                             clouds 1..L-1
// where cloud l+1 is level l's samples in ascending frame index (built by the
// gather kernel) and out_l the level's sample indices relative to cloud l.
// Its results (every level's samples as frame indices) are written by the
// gather kernel straight into its page-locked result slot, over the C2C link,
// and its frame comes in by one copy kernel per step that reads the
// page-locked frames of every admitted request: a step costs a few launches,
// not a copy call per request.
// When a step runs every level (the default), a request is admitted and
// finished within one step, so consecutive steps share no request: steps
// alternate between two streams (the caller's context and stream, and a
// second context of the runtime's own), and one step's frame copy over the
// C2C link overlaps the previous step's sampling on the SMs.
// Blocks start on 48-byte boundaries so that every xyz part starts on a point
// boundary of the arena (point offsets = byte offsets / 12) and every int32
// part on a 4-byte one.
#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <deque>
#include <map>
#include <memory>
#include <unordered_map>
#include <unordered_set>
#include <vector>

#include "../../include/afps.h"
#include "afps_internal.h"
#include "afps_trace.h"

namespace afps {
// afps_api.cu: reserve the context's shared workspace for tables of `bytes`.
int reserve_workspace(afps_ctx* ctx, size_t bytes);
}  // namespace afps

namespace {

constexpr int64_t kBlockAlign = 48;

struct Block {
    int64_t off = -1;  // bytes from the arena base
    int64_t bytes = 0;
};

// First-fit allocator over the arena with coalescing frees.
class Arena {
   public:
    explicit Arena(int64_t size) { free_[0] = size; }
    Block alloc(int64_t bytes) {
        bytes = (bytes + kBlockAlign - 1) / kBlockAlign * kBlockAlign;
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                Block b{it->first, bytes};
                const int64_t rest = it->second - bytes;
                const int64_t at = it->first + bytes;
                free_.erase(it);
                if (rest > 0) free_[at] = rest;
                used_ += bytes;
                return b;
            }
        }
        return Block{};
    }
    void release(const Block& b) {
        if (b.off < 0) return;
        used_ -= b.bytes;
        auto it = free_.emplace(b.off, b.bytes).first;
        auto next = std::next(it);
        if (next != free_.end() && it->first + it->second == next->first) {
            it->second += next->second;
            free_.erase(next);
        }
        if (it != free_.begin()) {
            auto prev = std::prev(it);
            if (prev->first + prev->second == it->first) {
                prev->second += it->second;
                free_.erase(it);
            }
        }
    }
    int64_t used() const { return used_; }

   private:
    std::map<int64_t, int64_t> free_;
    int64_t used_ = 0;
};

enum State { QUEUED, ACTIVE, COMPLETING, DONE, CANCELLED };

struct Request {
    uint64_t tag = 0;
    int64_t N = 0;
    Block staged;              // the frame in the page-locked pool until admitted
    const float* borrowed = nullptr;  // or the caller's page-locked frame (submit_pinned)
    const void* src_dev = nullptr;    // the frame's device-visible address (either case)
    State state = QUEUED;
    int level = 0;             // next level to sample
    Block block;
    int slot = -1;             // pinned result slot
    int lane = 0;              // the stream (and context) its work runs on
    int64_t xyz_pt[AFPS_SERVER_MAX_LEVELS + 1];  // cloud l, in points from the arena base
    int64_t out_el[AFPS_SERVER_MAX_LEVELS];      // out_l, in int32 elements
    int64_t fidx_el[AFPS_SERVER_MAX_LEVELS + 1]; // frame index of cloud l (l >= 1)
    cudaEvent_t done_ev = nullptr;
    double t_submit = 0, t_admit = 0, t_done = 0;
};

}  // namespace

struct afps_server {
    afps_ctx* ctx = nullptr;  // the caller's: lane 0
    afps_server_config cfg{};
    int levels[AFPS_SERVER_MAX_LEVELS] = {};
    int64_t total_samples = 0;  // sum of levels
    cudaStream_t stream = nullptr;  // lane 0
    bool own_stream = false;
    // steps alternate over `lanes` (stream, context) pairs: lane 0 is
    // (ctx, stream), lane 1 a stream and a clone of ctx owned here
    int lanes = 1;
    cudaStream_t lane_stream[2] = {};
    afps_ctx* lane_ctx[2] = {};
    uint64_t steps_run = 0;
    int device = 0;
    unsigned char* arena_base = nullptr;
    std::unique_ptr<Arena> arena;
    unsigned char* pool_base = nullptr;  // page-locked staging of queued frames
    std::unique_ptr<Arena> pool;
    // pool blocks whose host->device copy was issued in a step, with that
    // step's event: they are free once the event completes
    std::deque<std::pair<cudaEvent_t, std::vector<Block>>> pool_pending;
    int32_t* pinned = nullptr;  // max_inflight result slots
    int32_t* pinned_dev = nullptr;  // their device-visible address
    unsigned char* pool_dev = nullptr;  // device-visible address of the staging pool
    std::vector<int> free_slots;
    std::deque<std::unique_ptr<Request>> queue;
    std::vector<std::unique_ptr<Request>> active;  // ACTIVE or COMPLETING
    std::vector<std::unique_ptr<Request>> done;    // DONE, not yet polled
    std::vector<std::unique_ptr<Request>> handed;  // returned by the last poll
    std::deque<cudaEvent_t> step_events;           // steps in flight
    std::vector<cudaEvent_t> event_pool;
    // completion events shared by the requests that finished in one step:
    // the number of requests still holding each
    std::unordered_map<cudaEvent_t, int> ev_refs;
    std::chrono::steady_clock::time_point t0;
    double now() const {
        return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
            .count();
    }
};

namespace {

int64_t footprint(const afps_server* s, int64_t N) {
    int64_t pts = N, ints = 0;
    for (int l = 0; l < s->cfg.n_levels; ++l) {
        pts += s->levels[l];   // cloud l+1
        ints += s->levels[l];  // out_l
        if (l + 1 < s->cfg.n_levels) ints += s->levels[l];  // frame index of cloud l+1
    }
    return 12 * pts + 4 * ints + kBlockAlign;
}

cudaEvent_t take_event(afps_server* s) {
    if (!s->event_pool.empty()) {
        cudaEvent_t e = s->event_pool.back();
        s->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void give_event(afps_server* s, cudaEvent_t e) {
    if (e) s->event_pool.push_back(e);
}

// A request lets go of its completion event: a shared one returns to the
// pool with its last holder.
void drop_event(afps_server* s, cudaEvent_t e) {
    auto it = s->ev_refs.find(e);
    if (it != s->ev_refs.end() && --it->second > 0) return;
    if (it != s->ev_refs.end()) s->ev_refs.erase(it);
    give_event(s, e);
}

// Finished requests: the device work of their last step has completed.
void reap(afps_server* s) {
    // requests that finished in one step share its event: query each once
    cudaEvent_t last = nullptr;
    bool last_done = false;
    auto complete = [&](cudaEvent_t e) {
        if (e != last) {
            last = e;
            last_done = cudaEventQuery(e) == cudaSuccess;
        }
        return last_done;
    };
    for (auto& r : s->active) {
        if (r && r->state == COMPLETING && complete(r->done_ev)) {
            r->state = DONE;
            r->t_done = s->now();
            s->arena->release(r->block);
            r->block = Block{};
            drop_event(s, r->done_ev);
            r->done_ev = nullptr;
            s->done.push_back(std::move(r));
        } else if (r && r->state == CANCELLED && complete(r->done_ev)) {
            // no launched step uses its memory any more: drop it
            s->arena->release(r->block);
            drop_event(s, r->done_ev);
            s->free_slots.push_back(r->slot);
            r.reset();
        }
    }
    s->active.erase(std::remove(s->active.begin(), s->active.end(), nullptr), s->active.end());
    cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error here
}

bool admit_one(afps_server* s, Request& r) {
    if (s->free_slots.empty()) return false;
    Block b = s->arena->alloc(footprint(s, r.N));
    if (b.off < 0) return false;
    r.block = b;
    r.slot = s->free_slots.back();
    s->free_slots.pop_back();
    const int L = s->cfg.n_levels;
    int64_t pt = b.off / 12;  // b.off is a multiple of 48
    r.xyz_pt[0] = pt;
    pt += r.N;
    for (int l = 0; l < L; ++l) {
        r.xyz_pt[l + 1] = pt;
        pt += s->levels[l];
    }
    int64_t el = pt * 3;  // int32 elements after the xyz part
    for (int l = 0; l < L; ++l) {
        r.out_el[l] = el;
        el += s->levels[l];
    }
    r.fidx_el[0] = -1;
    for (int l = 1; l < L; ++l) {
        r.fidx_el[l] = el;
        el += s->levels[l - 1];
    }
    r.state = ACTIVE;
    r.level = 0;
    r.t_admit = s->now();
    return true;
}

}  // namespace

extern "C" {

int afps_server_create(afps_server** out, afps_ctx* ctx, const afps_server_config* cfg,
                       void* stream) {
    if (!out || !ctx || !cfg) return AFPS_ERR_INVALID_ARG;
    *out = nullptr;
    if (cfg->n_levels < 1 || cfg->n_levels > AFPS_SERVER_MAX_LEVELS || cfg->M < 1 ||
        cfg->npdu_window < 0 || cfg->hbm_budget_bytes <= 0)
        return AFPS_ERR_INVALID_ARG;
    for (int l = 0; l < cfg->n_levels; ++l) {
        if (cfg->levels[l] < 1 || cfg->levels[l] >= 65536) return AFPS_ERR_INVALID_ARG;
        if (l > 0 && cfg->levels[l] > cfg->levels[l - 1]) return AFPS_ERR_INVALID_ARG;
    }
    std::unique_ptr<afps_server> s(new (std::nothrow) afps_server());
    if (!s) return AFPS_ERR_NO_MEMORY;
    s->ctx = ctx;
    s->cfg = *cfg;
    if (s->cfg.max_inflight <= 0) s->cfg.max_inflight = 256;
    if (s->cfg.max_queued <= 0) s->cfg.max_queued = 4096;
    if (s->cfg.max_steps_ahead <= 0) s->cfg.max_steps_ahead = 2;
    for (int l = 0; l < cfg->n_levels; ++l) {
        s->levels[l] = cfg->levels[l];
        s->total_samples += cfg->levels[l];
    }
    s->t0 = std::chrono::steady_clock::now();
    if (cudaGetDevice(&s->device) != cudaSuccess) return AFPS_ERR_CUDA;
    if (stream) {
        s->stream = static_cast<cudaStream_t>(stream);
    } else {
        if (cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking) != cudaSuccess)
            return AFPS_ERR_CUDA;
        s->own_stream = true;
    }
    void* p = nullptr;
    if (cudaMalloc(&p, (size_t)cfg->hbm_budget_bytes) != cudaSuccess) {
        cudaGetLastError();
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return AFPS_ERR_NO_MEMORY;
    }
    s->arena_base = static_cast<unsigned char*>(p);
    s->arena.reset(new Arena(cfg->hbm_budget_bytes / kBlockAlign * kBlockAlign));
    void* h = nullptr;
    if (cudaMallocHost(&h, (size_t)s->cfg.max_inflight * s->total_samples * sizeof(int32_t)) !=
        cudaSuccess) {
        cudaGetLastError();
        cudaFree(p);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return AFPS_ERR_NO_MEMORY;
    }
    s->pinned = static_cast<int32_t*>(h);
    void* hd = nullptr;
    if (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess || !hd) {
        cudaGetLastError();
        cudaFreeHost(h);
        cudaFree(p);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return AFPS_ERR_CUDA;  // page-locked memory not mapped into the device
    }
    s->pinned_dev = static_cast<int32_t*>(hd);
    for (int i = s->cfg.max_inflight - 1; i >= 0; --i) s->free_slots.push_back(i);
    if (s->cfg.host_pool_bytes <= 0) s->cfg.host_pool_bytes = 64ll << 20;
    void* hp = nullptr;
    if (cudaMallocHost(&hp, (size_t)s->cfg.host_pool_bytes) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeHost(h);
        cudaFree(p);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return AFPS_ERR_NO_MEMORY;
    }
    s->pool_base = static_cast<unsigned char*>(hp);
    void* hpd = nullptr;
    if (cudaHostGetDevicePointer(&hpd, hp, 0) != cudaSuccess || !hpd) {
        cudaGetLastError();
        cudaFreeHost(hp);
        cudaFreeHost(h);
        cudaFree(p);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return AFPS_ERR_CUDA;
    }
    s->pool_dev = static_cast<unsigned char*>(hpd);
    s->pool.reset(new Arena(s->cfg.host_pool_bytes / kBlockAlign * kBlockAlign));
    // the largest step table: every slot's request at its widest level
    int32_t widest = 1;
    for (int l = 0; l < s->cfg.n_levels; ++l) widest = std::max(widest, std::min(s->cfg.M, s->levels[l]));
    const size_t table = std::max((size_t)s->cfg.max_inflight * widest * sizeof(afps::ItemDesc),
                                  (size_t)s->cfg.max_inflight * sizeof(afps::GatherDesc));
    const int rc = afps::reserve_workspace(ctx, table);
    if (rc != AFPS_OK) {
        cudaFreeHost(hp);
        cudaFreeHost(h);
        cudaFree(p);
        if (s->own_stream) cudaStreamDestroy(s->stream);
        return rc;
    }
    s->lane_stream[0] = s->stream;
    s->lane_ctx[0] = ctx;
    // a second lane when every step runs all levels (no request spans two
    // steps); without its stream or context the server runs on one
    const bool all_levels = s->cfg.levels_per_step <= 0 || s->cfg.levels_per_step >= s->cfg.n_levels;
    if (all_levels && afps::clone_context(ctx, &s->lane_ctx[1]) == AFPS_OK) {
        if (cudaStreamCreateWithFlags(&s->lane_stream[1], cudaStreamNonBlocking) == cudaSuccess &&
            afps::reserve_workspace(s->lane_ctx[1], table) == AFPS_OK) {
            s->lanes = 2;
        } else {
            cudaGetLastError();
            if (s->lane_stream[1]) cudaStreamDestroy(s->lane_stream[1]);
            afps_destroy(s->lane_ctx[1]);
            s->lane_stream[1] = nullptr;
            s->lane_ctx[1] = nullptr;
        }
    }
    *out = s.release();
    return AFPS_OK;
}

int afps_server_submit(afps_server* s, const float* h_xyz, int64_t N, uint64_t tag) {
    AFPS_TRACE("afps_server_submit");
    if (!s || !h_xyz || N < s->levels[0] || N > 65536) return AFPS_ERR_INVALID_ARG;
    if (footprint(s, N) > s->cfg.hbm_budget_bytes) return AFPS_ERR_INVALID_ARG;
    if ((int64_t)s->queue.size() >= s->cfg.max_queued) return AFPS_ERR_BUSY;
    // release staging blocks whose copies have completed
    while (!s->pool_pending.empty() && cudaEventQuery(s->pool_pending.front().first) == cudaSuccess) {
        for (const Block& b : s->pool_pending.front().second) s->pool->release(b);
        give_event(s, s->pool_pending.front().first);
        s->pool_pending.pop_front();
    }
    cudaGetLastError();
    const Block staged = s->pool->alloc(12 * N);
    if (staged.off < 0) return AFPS_ERR_BUSY;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) {
        s->pool->release(staged);
        return AFPS_ERR_NO_MEMORY;
    }
    r->tag = tag;
    r->N = N;
    r->staged = staged;
    r->src_dev = s->pool_dev + staged.off;
    memcpy(s->pool_base + staged.off, h_xyz, (size_t)(12 * N));
    r->t_submit = s->now();
    s->queue.push_back(std::move(r));
    return AFPS_OK;
}

int afps_server_submit_pinned(afps_server* s, const float* h_xyz, int64_t N, uint64_t tag) {
    AFPS_TRACE("afps_server_submit_pinned");
    if (!s || !h_xyz || N < s->levels[0] || N > 65536) return AFPS_ERR_INVALID_ARG;
    if (footprint(s, N) > s->cfg.hbm_budget_bytes) return AFPS_ERR_INVALID_ARG;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, h_xyz) != cudaSuccess || at.type != cudaMemoryTypeHost ||
        !at.devicePointer || reinterpret_cast<uintptr_t>(at.devicePointer) % 4) {
        cudaGetLastError();
        return AFPS_ERR_INVALID_ARG;
    }
    if ((int64_t)s->queue.size() >= s->cfg.max_queued) return AFPS_ERR_BUSY;
    std::unique_ptr<Request> r(new (std::nothrow) Request());
    if (!r) return AFPS_ERR_NO_MEMORY;
    r->tag = tag;
    r->N = N;
    r->borrowed = h_xyz;
    r->src_dev = at.devicePointer;
    r->t_submit = s->now();
    s->queue.push_back(std::move(r));
    return AFPS_OK;
}

int afps_server_cancel(afps_server* s, uint64_t tag) {
    AFPS_TRACE("afps_server_cancel");
    if (!s) return AFPS_ERR_INVALID_ARG;
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it) {
        if ((*it)->tag == tag) {  // not admitted: nothing on the device yet
            s->pool->release((*it)->staged);
            s->queue.erase(it);
            return AFPS_OK;
        }
    }
    for (auto& r : s->active) {
        if (r && r->tag == tag && r->state == ACTIVE) {
            // later steps leave it out; its memory is freed once every step
            // launched so far (all before this event) has completed
            cudaEvent_t e = take_event(s);
            if (!e) return AFPS_ERR_CUDA;
            if (cudaEventRecord(e, s->lane_stream[r->lane]) != cudaSuccess) {
                cudaGetLastError();
                give_event(s, e);
                return AFPS_ERR_CUDA;
            }
            r->state = CANCELLED;
            r->done_ev = e;
            return AFPS_OK;
        }
    }
    return AFPS_ERR_INVALID_ARG;
}

int afps_server_step(afps_server* s) {
    AFPS_TRACE("afps_server_step");
    if (!s) return AFPS_ERR_INVALID_ARG;
    // stay at most max_steps_ahead steps ahead of the GPU
    while ((int)s->step_events.size() >= s->cfg.max_steps_ahead) {
        cudaEvent_t e = s->step_events.front();
        s->step_events.pop_front();
        cudaError_t err = cudaEventSynchronize(e);
        give_event(s, e);
        if (err != cudaSuccess) return AFPS_ERR_CUDA;
    }
    while (!s->step_events.empty() && cudaEventQuery(s->step_events.front()) == cudaSuccess) {
        give_event(s, s->step_events.front());
        s->step_events.pop_front();
    }
    cudaGetLastError();
    reap(s);

    // this step's lane (stream and context)
    const int lane = (int)(s->steps_run % (uint64_t)s->lanes);
    cudaStream_t st = s->lane_stream[lane];
    afps_ctx* cx = s->lane_ctx[lane];

    // admission, first come first served, by arena footprint and slots
    float* xyz = reinterpret_cast<float*>(s->arena_base);
    int32_t* ints = reinterpret_cast<int32_t*>(s->arena_base);
    std::vector<Block> copied;  // staging blocks read by this step's copies
    afps::FrameCopyBatch batch;
    batch.n = 0;
    int64_t batch_max = 0;
    auto flush = [&]() -> bool {
        const bool ok = afps::launch_frame_copy(batch, batch_max, st) == cudaSuccess;
        batch.n = 0;
        batch_max = 0;
        return ok;
    };
    while (!s->queue.empty() && (int)s->active.size() < s->cfg.max_inflight) {
        Request& r = *s->queue.front();
        if (!admit_one(s, r)) break;
        r.lane = lane;
        batch.c[batch.n++] = afps::FrameCopy{r.src_dev, xyz + 3 * r.xyz_pt[0], 12 * r.N};
        batch_max = std::max(batch_max, 12 * r.N);
        if (batch.n == afps::kFrameCopyMax && !flush()) {
            cudaGetLastError();
            return AFPS_ERR_CUDA;
        }
        if (!r.borrowed) copied.push_back(r.staged);
        r.staged = Block{};
        s->active.push_back(std::move(s->queue.front()));
        s->queue.pop_front();
    }
    if (batch.n > 0 && !flush()) {
        cudaGetLastError();
        return AFPS_ERR_CUDA;
    }
    if (!copied.empty()) {
        cudaEvent_t ce = take_event(s);
        if (!ce || cudaEventRecord(ce, st) != cudaSuccess) return AFPS_ERR_CUDA;
        s->pool_pending.emplace_back(ce, std::move(copied));
    }

    // level after level: one batched sampling launch over every active
    // request's current level (mixed levels share it), then the gather
    const int per_step = s->cfg.levels_per_step > 0 ? s->cfg.levels_per_step : s->cfg.n_levels;
    int advanced = 0;
    for (int sub = 0; sub < per_step; ++sub) {
        // one batched sampling launch over every active request's current level
        std::vector<Request*> run;
        for (auto& r : s->active)
            if (r->state == ACTIVE) run.push_back(r.get());
        if (run.empty()) break;
        const int32_t B = (int32_t)run.size();
        std::vector<int64_t> pt_begin(B), n_pts(B), start(B, 0), out_begin(B);
        std::vector<int32_t> C(B), M(B), K(B, s->cfg.npdu_window);
        std::vector<afps::GatherDesc> g(B);
        for (int32_t b = 0; b < B; ++b) {
            Request& r = *run[b];
            const int l = r.level;
            const int64_t n = l == 0 ? r.N : s->levels[l - 1];
            pt_begin[b] = r.xyz_pt[l];
            n_pts[b] = n;
            C[b] = s->levels[l];
            M[b] = std::min(s->cfg.M, C[b]);
            out_begin[b] = r.out_el[l];
            afps::GatherDesc& d = g[b];
            d.in_xyz = r.xyz_pt[l];
            d.in_frame = r.fidx_el[l];  // -1 at level 0: the frame itself
            d.sel = r.out_el[l];
            d.out_xyz = r.xyz_pt[l + 1];
            d.out_frame = l + 1 < s->cfg.n_levels ? r.fidx_el[l + 1] : -1;
            int64_t res = (int64_t)r.slot * s->total_samples;  // in the result slot
            for (int q = 0; q < l; ++q) res += s->levels[q];
            d.sel_frame = res;
            d.n = (int32_t)n;
            d.c = C[b];
        }
        int rc = afps::sample_scattered(cx, xyz, B, pt_begin.data(), n_pts.data(), C.data(),
                                        M.data(), K.data(), start.data(), ints, out_begin.data(),
                                        st);
        if (rc == AFPS_OK)
            rc = afps::gather_run(cx, g.data(), B, xyz, ints, ints, xyz, ints, s->pinned_dev, st);
        if (rc != AFPS_OK) {
            afps::copy_error(s->ctx, cx);
            return rc;
        }

        // finished chains: their results are in their slots once the step's
        // gather has completed
        cudaEvent_t fin = nullptr;
        for (Request* r : run) {
            if (++r->level < s->cfg.n_levels) continue;
            r->state = COMPLETING;
            if (!fin) fin = take_event(s);
        }
        if (fin) {
            if (cudaEventRecord(fin, st) != cudaSuccess) return AFPS_ERR_CUDA;
            // the finishing requests share the step's completion event
            int holders = 0;
            for (Request* r : run) {
                if (r->state != COMPLETING || r->done_ev) continue;
                r->done_ev = fin;
                ++holders;
            }
            s->ev_refs[fin] = holders;
        }
        advanced += (int)run.size();
    }
    if (advanced == 0) return 0;
    cudaEvent_t se = take_event(s);
    if (!se || cudaEventRecord(se, st) != cudaSuccess) return AFPS_ERR_CUDA;
    s->step_events.push_back(se);
    ++s->steps_run;
    return advanced;
}

int afps_server_poll(afps_server* s, afps_server_result* out, int32_t max_results) {
    AFPS_TRACE("afps_server_poll");
    if (!s || (!out && max_results > 0)) return AFPS_ERR_INVALID_ARG;
    // results handed out by the previous poll give their slots back now
    for (auto& r : s->handed) s->free_slots.push_back(r->slot);
    s->handed.clear();
    reap(s);
    int n = 0;
    size_t k = 0;  // results taken from the front of `done`
    while (n < max_results && k < s->done.size()) {
        std::unique_ptr<Request> r = std::move(s->done[k++]);
        afps_server_result& o = out[n++];
        memset(&o, 0, sizeof(o));
        o.tag = r->tag;
        o.status = AFPS_OK;
        o.n_levels = s->cfg.n_levels;
        for (int l = 0; l < s->cfg.n_levels; ++l) o.count[l] = s->levels[l];
        o.indices = s->pinned + (int64_t)r->slot * s->total_samples;
        o.submit_ms = r->t_submit;
        o.admit_ms = r->t_admit;
        o.done_ms = r->t_done;
        s->handed.push_back(std::move(r));
    }
    s->done.erase(s->done.begin(), s->done.begin() + (std::ptrdiff_t)k);
    return n;
}

int afps_server_stats(afps_server* s, int64_t* queued, int64_t* inflight, int64_t* arena_used) {
    if (!s) return AFPS_ERR_INVALID_ARG;
    if (queued) *queued = (int64_t)s->queue.size();
    if (inflight) *inflight = (int64_t)s->active.size();
    if (arena_used) *arena_used = s->arena->used();
    return AFPS_OK;
}

double afps_server_clock_ms(const afps_server* s) { return s ? s->now() : 0.0; }

void afps_server_destroy(afps_server* s) {
    if (!s) return;
    cudaStreamSynchronize(s->stream);
    if (s->lane_stream[1]) cudaStreamSynchronize(s->lane_stream[1]);
    std::unordered_set<cudaEvent_t> held;  // shared events are destroyed once
    for (auto& r : s->active)
        if (r && r->done_ev) held.insert(r->done_ev);
    for (cudaEvent_t e : held) cudaEventDestroy(e);
    for (cudaEvent_t e : s->step_events) cudaEventDestroy(e);
    for (auto& pp : s->pool_pending) cudaEventDestroy(pp.first);
    if (s->pool_base) cudaFreeHost(s->pool_base);
    for (cudaEvent_t e : s->event_pool) cudaEventDestroy(e);
    if (s->arena_base) cudaFree(s->arena_base);
    if (s->pinned) cudaFreeHost(s->pinned);
    if (s->own_stream) cudaStreamDestroy(s->stream);
    if (s->lane_stream[1]) cudaStreamDestroy(s->lane_stream[1]);
    if (s->lane_ctx[1]) afps_destroy(s->lane_ctx[1]);
    cudaGetLastError();
    delete s;
}

}  // extern "C"
