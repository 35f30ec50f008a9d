// afps_device.cuh -- inline-PTX helpers for sm_103a: mbarriers, 1-D bulk
// copies (TMA engine), cluster shared memory and barriers, bounded waits.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "afps_internal.h"

namespace afps {
namespace dev {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Programmatic dependent launch: let the next kernel of the stream be
// scheduled before this one ends, and wait (before the first global memory
// access) until the previous kernel has completed and its writes are
// visible.  Both are no-ops for launches without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Hint: bring the 128-byte line holding p into L2.  No data is returned and
// nothing changes for coherence, so it may be issued before pdl_wait.
__device__ __forceinline__ void prefetch_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// ---------------------------------------------------------------- mbarrier
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// Make barrier initialisation visible to the async proxy (bulk copies) and to
// the other CTAs of a cluster.
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Order this thread's earlier generic-proxy shared-memory accesses before
// later async-proxy (bulk copy) accesses.
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile(
        "{\n\t.reg .b64 st;\n\t"
        "mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(bar),
        "r"(bytes)
        : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// As mbar_try_wait, with the thread suspended for up to hint_ns while the
// phase is incomplete (fewer polling instructions while a copy is in flight).
__device__ __forceinline__ bool mbar_try_wait_for(uint32_t bar, uint32_t parity,
                                                  uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}

// Wait for phase `parity` of the barrier to complete, giving up after
// timeout_ns.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity,
                                                  uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait_for(bar, parity, 20000u)) return true;
        if (globaltimer() - t0 > timeout_ns) return false;
    }
}

// 1-D bulk copy global -> shared, completion signalled on `bar` as bytes.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, "
        "[%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

// ---------------------------------------------------------------- clusters
__device__ __forceinline__ uint32_t cluster_ctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_nctarank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_nctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t cluster_id_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
    return r;
}
__device__ __forceinline__ uint32_t ncluster_x() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%nclusterid.x;" : "=r"(r));
    return r;
}
// Address of the same shared-memory offset in CTA `rank` of this cluster.
__device__ __forceinline__ uint32_t mapa(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint32_t a, uint32_t b,
                                              uint32_t c, uint32_t d) {
    asm volatile("st.shared::cluster.v4.u32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a),
                 "r"(b), "r"(c), "r"(d)
                 : "memory");
}
// Asynchronous 16-byte store into another CTA's shared memory whose
// completion is counted (as bytes) on that CTA's mbarrier `remote_bar`.
__device__ __forceinline__ void st_async_v4(uint32_t remote_addr, uint32_t remote_bar, uint32_t a,
                                            uint32_t b, uint32_t c, uint32_t d) {
    asm volatile(
        "st.async.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%2, %3, %4, %5}, "
        "[%1];" ::"r"(remote_addr),
        "r"(remote_bar), "r"(a), "r"(b), "r"(c), "r"(d)
        : "memory");
}
// Full cluster barrier with release/acquire ordering of shared::cluster memory.
__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
    asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// ---------------------------------------------------------------- misc
__device__ __forceinline__ void record_status(int* status, int code) {
    if (status) atomicCAS(status, 0, code);
}

// Whether the status word holds a timeout (any launch on the context since
// the last afps_sync).  A volatile load: issued where it stands, so it can be
// placed ahead of a wait and its latency hidden behind it.
__device__ __forceinline__ int load_status(const int* status) {
    int v = 0;
    if (status) asm volatile("ld.volatile.global.s32 %0, [%1];" : "=r"(v) : "l"(status) : "memory");
    return v;
}
__device__ __forceinline__ bool is_timeout(int status) {
    return status == DEV_TIMEOUT_STAGE || status == DEV_TIMEOUT_DRAIN ||
           status == DEV_TIMEOUT_EXCHANGE;
}

// Next item of a dynamic work queue (one ticket per warp, drawn by lane 0).
// Every warp of the grid draws tickets until one lies past the last item, so
// a launch draws exactly n_items + (warps in the grid) tickets; the warp that
// draws the last of them is the last to touch the counter and sets it back
// to zero for the next launch (no memset between launches).
__device__ __forceinline__ int queue_next_of(unsigned* counter, int n, int nwarps, int lane) {
    unsigned v = 0;
    if (lane == 0) {
        v = atomicAdd(counter, 1u);
        if (v == (unsigned)n + (unsigned)nwarps - 1u) atomicExch(counter, 0u);
    }
    return (int)__shfl_sync(kFull, v, 0);
}
__device__ __forceinline__ int queue_next(const LaunchArgs& a, int nwarps, int lane) {
    return queue_next_of(a.counter, a.n_items, nwarps, lane);
}

// Debug build (AFPS_DEBUG_CHECKS): index v must lie in [lo, hi); otherwise
// the failure is recorded and v is clamped into the range, so the access it
// guards stays in bounds.  The regular build returns v unchanged.
__device__ __forceinline__ int checked(int v, int lo, int hi, int* status) {
#ifdef AFPS_DEBUG_CHECKS
    if (v < lo || v >= hi) {
        record_status(status, DEV_CHECK_FAILED);
        return v < lo ? lo : hi - 1;
    }
#endif
    (void)lo;
    (void)hi;
    (void)status;
    return v;
}

// Squared distance with every product and sum rounded on its own (the
// intrinsics are never contracted into fused multiply-adds).
__device__ __forceinline__ float sqdist(float x, float y, float z, float qx, float qy,
                                        float qz) {
    const float dx = __fsub_rn(x, qx);
    const float dy = __fsub_rn(y, qy);
    const float dz = __fsub_rn(z, qz);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Two fp32 lanes in one 64-bit register, for the packed f32x2 arithmetic of
// sm_100-class GPUs: each lane is rounded exactly like the scalar operation.
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}

__device__ __forceinline__ void unpack2(unsigned long long r, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(r));
}

// Squared distances of two points (packed x, y, z) to q (q broadcast in both
// lanes): the same separately rounded (dx*dx + dy*dy) + dz*dz as sqdist.  The
// differences and squares use packed f32x2 instructions; the two sums are
// scalar .rn adds, because a packed add that follows packed products may be
// fused with them into a single rounding, while scalar adds with an explicit
// rounding mode are never fused (a one-ulp difference was measured on a
// 16K-point cloud with packed adds).
__device__ __forceinline__ void sqdist2(unsigned long long x, unsigned long long y,
                                       unsigned long long z, unsigned long long qx,
                                       unsigned long long qy, unsigned long long qz, float& d0,
                                       float& d1) {
    unsigned long long dx, dy, dz;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(x), "l"(qx));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(y), "l"(qy));
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(z), "l"(qz));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(dx) : "l"(dx), "l"(dx));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(dy) : "l"(dy), "l"(dy));
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(dz) : "l"(dz), "l"(dz));
    float x0, x1, y0, y1, z0, z1;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(x0), "=f"(x1) : "l"(dx));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(y0), "=f"(y1) : "l"(dy));
    asm("mov.b64 {%0, %1}, %2;" : "=f"(z0), "=f"(z1) : "l"(dz));
    d0 = __fadd_rn(__fadd_rn(x0, y0), z0);
    d1 = __fadd_rn(__fadd_rn(x1, y1), z1);
}

// Unsigned division of x < 2^24 by a divisor d >= 1 used many times: the
// product of x and the rounded reciprocal is within (x/d) 2^-23 < 1 of x/d
// for d >= 2 (exact for d = 1), so its truncation is the quotient or one off
// either way, which two integer checks correct.
struct SmallDiv {
    uint32_t d;
    float r;
    __device__ __forceinline__ explicit SmallDiv(uint32_t dd) : d(dd), r(1.0f / (float)dd) {}
    __device__ __forceinline__ uint32_t operator()(uint32_t x) const {
        uint32_t t = __float2uint_rz(__uint2float_rn(x) * r);
        t -= t * d > x ? 1u : 0u;
        t += (t + 1u) * d <= x ? 1u : 0u;
        return t;
    }
};

// Item `i` of a launch: from the device table, or computed (cloud i / M,
// sector i % M) with the sector rule floor(s*N/M), floor(s*C/M) from the
// parameters of a run of equal clouds stored back to back, or from the
// cloud's record (offsets, N, C).  Back to back no memory is read at all
// ahead of the stage-in; with records the host builds one per cloud instead
// of M table entries.
__device__ __forceinline__ ItemDesc load_item(const LaunchArgs& a, int i) {
    if (a.items) return a.items[i];
    const SingleCloud& s = a.single;
    const uint32_t M = (uint32_t)s.M;
    const uint64_t mm = s.m_magic;
    // x / M for x < 2^32 by one multiply-high (div_magic), or a division when M < 2
    auto divM = [M, mm](uint32_t x) -> uint32_t {
        return mm ? (uint32_t)__umul64hi((uint64_t)x, mm) : x / M;
    };
    const uint32_t b = divM((uint32_t)i);
    const uint32_t sec = (uint32_t)i - b * M;
    int32_t N = s.N, C = s.C;
    int64_t src0, dst0;
    if (s.clouds) {
        const CloudRec r = s.clouds[b];
        N = r.N;
        C = r.C;
        src0 = r.pt_off;
        dst0 = r.out_off;
    } else {
        src0 = s.pt_off + (int64_t)b * N;
        dst0 = s.out_off + (int64_t)b * C;
    }
    int64_t lo, hi, o0, o1;
    if (s.wide) {  // M * N does not fit in 32 bits
        lo = (int64_t)sec * N / s.M;
        hi = (int64_t)(sec + 1) * N / s.M;
        o0 = (int64_t)sec * C / s.M;
        o1 = (int64_t)(sec + 1) * C / s.M;
    } else {  // numerators below M * N < 2^32
        lo = divM(sec * (uint32_t)N);
        hi = divM((sec + 1) * (uint32_t)N);
        o0 = divM(sec * (uint32_t)C);
        o1 = divM((sec + 1) * (uint32_t)C);
    }
    ItemDesc d;
    d.src = src0 + lo;
    d.dst = dst0 + o0;
    d.n = (int32_t)(hi - lo);
    d.c = (int32_t)(o1 - o0);
    d.first = s.start_r < d.n - 1 ? s.start_r : d.n - 1;
    d.lo = (int32_t)lo;
    d.kl = s.kl;
    d.kr = s.kr;
    d.flags = s.flags;
    d.pad = 0;
    return d;
}

// Stage n points (3 floats each, starting at g, 4-byte aligned) into the
// 16-byte aligned shared buffer `buf` (capacity >= 12 n + 16 bytes).  The
// 16-byte aligned interior goes by one bulk copy issued by `issuer` and
// completing on `bar`; the unaligned head and tail (at most 3 floats each)
// are plain loads spread over threads tid = 0 .. nthr-1.  `stall` (fault
// injection) arms the barrier without issuing the copy.  `no_bulk` stages
// everything with plain loads (points in host memory reached over the C2C
// link, which the bulk-copy engine is not used for).  Returns the shared
// address of point 0 and sets *bulk when a bulk copy was issued (the caller
// then waits for the barrier's phase and synchronises its threads).
__device__ __forceinline__ float* stage_points(const float* g, int n, unsigned char* buf,
                                               uint32_t bar, bool issuer, int tid, int nthr,
                                               bool* bulk, bool stall = false,
                                               bool no_bulk = false) {
    const uintptr_t A = reinterpret_cast<uintptr_t>(g);
    const uintptr_t E = A + 12ull * (uint64_t)n;
    const uintptr_t a0 = A & ~uintptr_t(15);
    const uintptr_t i0 = (A + 15) & ~uintptr_t(15);
    const uintptr_t i1 = E & ~uintptr_t(15);
    float* s = reinterpret_cast<float*>(buf + (A - a0));
    const bool use_bulk = i1 > i0 && !no_bulk;
    int nh, ts;
    if (use_bulk) {
        nh = (int)((i0 - A) >> 2);
        ts = (int)((i1 - A) >> 2);
        if (issuer) {
            mbar_arrive_expect_tx(bar, (uint32_t)(i1 - i0));
            if (!stall)
                bulk_g2s(smem_u32(buf + (i0 - a0)), reinterpret_cast<const void*>(i0),
                         (uint32_t)(i1 - i0), bar);
        }
    } else {
        nh = 3 * n;
        ts = 3 * n;
    }
    for (int f = tid; f < nh; f += nthr) s[f] = g[f];
    for (int f = ts + tid; f < 3 * n; f += nthr) s[f] = g[f];
    *bulk = use_bulk;
    return s;
}

}  // namespace dev
}  // namespace afps
