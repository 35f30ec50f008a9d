// afps_cta.cu -- one CTA, or one thread-block cluster of CS CTAs, per sector.
//
// Used for sectors larger than a warp holds in registers, and for plain FPS
// (M = 1) on whole clouds: the cross-core argmax that Sec. III-B calls the
// scaling limit of parallel FPS.  The sector is split into CS contiguous
// chunks, one per CTA; each CTA stages its chunk into shared memory by bulk
// copy and thread t keeps chunk points t + T i (i < P) in registers.
//
// One iteration = one CTA barrier:
//   1. update + local argmax in registers (all points, or the NPDU window);
//   2. warp argmax (two redux.sync steps) to a key {distance bits, ~index}.
//      CS == 1: lane 0 stores the key as the warp's record, then bar.sync.
//      CS > 1: the warps' keys meet in shared memory; behind a bar.sync
//      warp 0 reduces them to the CTA's record and its lanes 0..CS-1 store
//      that record, with the winning point's x, y, z, into slot `rank` of
//      every CTA of the cluster (itself included) by st.async, whose bytes
//      complete a transaction count on the receiving CTA's mbarrier (one per
//      record buffer).  One record per CTA keeps each mbarrier at CS
//      transfers per exchange; every thread then waits on its own CTA's
//      mbarrier, which is cheaper than a cluster barrier.  The buffer of the
//      previous exchange is re-armed behind the same bar.sync (all its
//      readers have passed it), before this CTA's records can let a peer
//      start the next exchange;
//   3. every warp reduces the exchange's records itself (a lane per record,
//      then redux.sync), which yields the next sample without a second
//      barrier; its coordinates come from this CTA's shared memory (CS == 1)
//      or from its owner CTA's record (CS > 1).  Records are double-buffered
//      by exchange parity, so a record is never overwritten before every
//      reader passed the barrier that follows its read.
#include <map>
#include <mutex>
#include <set>
#include <utility>

#include "afps_device.cuh"

namespace afps {

struct __align__(16) Rec {
    uint32_t bits;  // distance bits of the candidate (>= +0)
    uint32_t jinv;  // 0xffffffff - sector index: larger = lower index
    float x, y, z;
    uint32_t pad[3];
};
static_assert(sizeof(Rec) == 32, "Rec layout");

// Wait for an exchange's records: polls mbarrier.test_wait (no suspension)
// and reads the clock every 32 polls, giving up after timeout_ns.  While an
// exchange is pending every warp of the CTA waits on it, so polling takes no
// issue slot from useful work, and the records are seen as soon as they land.
__device__ __forceinline__ bool exchange_wait(uint32_t bar, uint32_t parity, uint64_t timeout_ns) {
    auto test = [&]() {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(parity)
            : "memory");
        return ok != 0;
    };
    if (test()) return true;
    const uint64_t t0 = dev::globaltimer();
    while (true) {
        for (int k = 0; k < 32; ++k)
            if (test()) return true;
        if (dev::globaltimer() - t0 > timeout_ns) return false;
    }
}

template <int P, bool NPDU, bool CLUSTER>
__global__ void __launch_bounds__(P >= 16 ? 256 : 1024) afps_cta_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int T = blockDim.x;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int w = tid >> 5;
    const int W = T >> 5;
    const int CS = CLUSTER ? (int)dev::cluster_nctarank() : 1;
    const int rank = CLUSTER ? (int)dev::cluster_ctarank() : 0;
    // records per exchange buffer: one per CTA of the cluster, or one per
    // warp of the CTA
    const int E = CLUSTER ? CS : W;

    // [stage-in barrier | exchange barriers x2 | pad] [records 2 x E]
    // [cluster: the warps' keys, W x 8 bytes, padded to 16] [points]
    uint64_t* barp = reinterpret_cast<uint64_t*>(smem);
    Rec* recs = reinterpret_cast<Rec*>(smem + 32);
    uint2* wkeys = reinterpret_cast<uint2*>(smem + 32 + 2 * E * sizeof(Rec));
    unsigned char* buf =
        smem + 32 + 2 * E * sizeof(Rec) + (CLUSTER ? 16 * ((8 * W + 15) / 16) : 0);
    const uint32_t bar = dev::smem_u32(barp);
    const uint32_t xbar0 = dev::smem_u32(barp + 1), xbar1 = dev::smem_u32(barp + 2);
    const uint32_t xbytes = (uint32_t)(E * sizeof(Rec));  // expected per exchange
    if (tid == 0) {
        dev::mbar_init(bar, 1);
        if (CLUSTER) {
            dev::mbar_init(xbar0, 1);
            dev::mbar_init(xbar1, 1);
        }
        dev::fence_mbar_init();
        if (CLUSTER) {
            dev::mbar_arrive_expect_tx(xbar0, xbytes);
            dev::mbar_arrive_expect_tx(xbar1, xbytes);
        }
    }
    __syncthreads();
    if (CLUSTER) dev::cluster_sync();  // every peer's barriers exist before any remote store
    // A computed first item (no table, no cloud records) needs no memory
    // access, so this CTA's part of its points can be prefetched into L2
    // while the previous kernel of the stream still runs.
    {
        const int g0 = CLUSTER ? (int)dev::cluster_id_x() : (int)blockIdx.x;
        if (!a.items && !a.single.clouds && !a.host_resident && g0 < a.n_items) {
            const ItemDesc d0 = dev::load_item(a, g0);
            const int ch = CLUSTER ? (d0.n + CS - 1) / CS : d0.n;
            const int p0 = rank * ch, pn = max(0, min(d0.n - p0, ch));
            const char* g = reinterpret_cast<const char*>(a.xyz + 3 * (d0.src + p0));
            for (int off = 128 * tid; off < 12 * pn; off += 128 * T) dev::prefetch_l2(g + off);
        }
    }
    // Programmatic dependent launch: wait until the previous kernel of the
    // stream has completed (no global memory access before this), then let
    // the next one be scheduled: one kernel waits behind a running one, and
    // the chain never grows deeper than that.
    dev::pdl_wait();
    dev::pdl_launch_dependents();
    // barrier addresses and phases in scalars: a two-element array indexed
    // by the exchange parity would live in a local-memory stack frame
    uint32_t xphase0 = 0u, xphase1 = 0u;

    uint32_t phase = 0;
    uint32_t xchg = 0;  // exchange counter: record buffer parity
    // cluster stride phase: every CTA's 1e10-test verdict, two alternating buffers
    __shared__ __align__(16) uint32_t cl_ok[CLUSTER ? 2 : 1][CLUSTER ? 16 : 1][4];
    uint32_t npro = 0;  // stride phases run (buffer parity)
    // cluster: every CTA's stop verdict of each item, two alternating buffers
    __shared__ __align__(16) uint32_t cl_stop[CLUSTER ? 2 : 1][CLUSTER ? 16 : 1][4];
    uint32_t nvote = 0;
    bool halted = false;  // a timeout was seen: leave the remaining items undone
    const int group = CLUSTER ? (int)dev::cluster_id_x() : (int)blockIdx.x;
    const int ngroups = CLUSTER ? (int)dev::ncluster_x() : (int)gridDim.x;

    for (int item = group; item < a.n_items; item += ngroups) {
        const ItemDesc d = dev::load_item(a, item);
        const int n = dev::checked(d.n, 1, CS * T * P + 1, a.status);  // fits the CTA(s)
        const int chunk = CLUSTER ? (n + CS - 1) / CS : n;
        const int c0 = rank * chunk;
        const int cn = max(0, min(n - c0, chunk));

        // ---- stage-in of this CTA's chunk
        dev::fence_proxy_async_smem();
        __syncthreads();
        bool bulk = false;
        bool late = false;
        int seen = 0;
        const float* pts = reinterpret_cast<const float*>(buf);
        if (cn > 0 && !halted)
            pts = dev::stage_points(a.xyz + 3 * (d.src + c0), cn, buf, bar, tid == 0, tid, T,
                                    &bulk, (a.stall & STALL_COPY) != 0, a.host_resident != 0);
        // a timeout recorded by any CTA so far (the load overlaps the copy)
        if (!halted) seen = dev::load_status(a.status);
        if (bulk) {
            late = !dev::mbar_wait_bounded(bar, phase, a.timeout_ns);
            if (late) {
                dev::record_status(a.status, DEV_TIMEOUT_STAGE);
                if (!dev::mbar_wait_bounded(bar, phase, a.timeout_ns))
                    dev::record_status(a.status, DEV_TIMEOUT_DRAIN);
            }
            phase ^= 1u;
        }
        // After a timeout (here, in a peer or anywhere on the context) nothing
        // is computed on shared memory a copy may not have filled.  The CTAs
        // of a cluster agree on it item by item (each CTA's verdict to every
        // peer, one cluster barrier), so they all skip the same items and
        // pass the same sequence of cluster barriers.
        bool stop = __syncthreads_or(halted || late || dev::is_timeout(seen)) != 0;
        if (CLUSTER) {
            const int par = nvote & 1;
            if (tid < CS)
                dev::st_cluster_v4(dev::mapa(dev::smem_u32(&cl_stop[par][rank][0]), (uint32_t)tid),
                                   stop ? 1u : 0u, 0u, 0u, 0u);
            dev::cluster_sync();
            for (int r = 0; r < CS; ++r) stop = stop || cl_stop[par][r][0] != 0u;
            ++nvote;
        }
        halted = stop;
        if (halted) continue;

        // rows i = 2h, 2h+1 share packed registers (f32x2 arithmetic)
        constexpr int PP = (P + 1) / 2;
        unsigned long long X2[PP], Y2[PP], Z2[PP];
        float D[2 * PP];
#pragma unroll
        for (int h = 0; h < PP; ++h) {
            float xs[2], ys[2], zs[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int i = 2 * h + u;
                const int jl = tid + T * i;
                if (i < P && jl < cn) {
                    xs[u] = pts[3 * jl];
                    ys[u] = pts[3 * jl + 1];
                    zs[u] = pts[3 * jl + 2];
                    D[i] = 1e10f;
                } else {  // padding: distance +0 stays +0 and loses every tie
                    xs[u] = 0.f;
                    ys[u] = 0.f;
                    zs[u] = 0.f;
                    D[i] = 0.f;
                }
            }
            X2[h] = dev::pack2(xs[0], xs[1]);
            Y2[h] = dev::pack2(ys[0], ys[1]);
            Z2[h] = dev::pack2(zs[0], zs[1]);
        }

        int p = dev::checked(d.first, 0, n, a.status);  // sector offset of the current sample
        const float* gq = a.xyz + 3 * (d.src + p);
        float qx = gq[0], qy = gq[1], qz = gq[2];
        int32_t* out = a.out + d.dst;
        const int c = dev::checked(d.c, 1, n + 1, a.status);
        const int kl = d.kl;
        const int kr = d.kr;
        const bool full_first = (d.flags & ITEM_FULL_FIRST) != 0;
        const bool emitter = (rank == 0) && (w == 0);
        int obuf = lane == 0 ? d.lo + p : 0;

        int t0 = 1;
        // (not in the 8-points-per-thread cluster kernel: at 1024 threads its
        // 64 registers leave no room, and the tuner has its neighbours)
        constexpr bool kStride = NPDU && !(CLUSTER && P == 8);
        if (kStride && !full_first && p <= kl && kl <= kr) {  // the same for every CTA of a cluster
            // Stride phase of the literal NPDU reading (Sec. III-C; distances
            // start at 1e10): while points past the last window are untouched
            // they hold the maximum, so the lowest-index argmax is the first of
            // them and the samples are p, p + q, p + 2q, ... (q = kr + 1) until
            // a window reaches the sector's end.  Their window updates run here
            // at once (with kl <= kr a point lies in at most two windows); the
            // argmax rounds they replace are decided in advance provided every
            // windowed distance is below 1e10, else the serial loop runs from
            // the start.  A cluster's CTAs each hold a chunk: the samples'
            // coordinates come from memory and the 1e10 test is combined
            // across the cluster.
            const int q = kr + 1;
            const int x = n - 1 - kr - p;
            const dev::SmallDiv divq((uint32_t)q);
            const int ts = x <= 0 ? 1 : (int)divq((uint32_t)(x + q - 1)) + 1;  // stride length
            const int tn = min(ts, c);                        // of them emitted
            const int tw = min(ts, c - 1);                    // whose window is applied
            const float* G = CLUSTER ? a.xyz + 3 * d.src : pts;  // the sector's points
            bool ok = true;  // D is updated in place and reset if the test fails
            // Window u = floor((j + kl - p) / q) is the last one starting at or
            // before point j and always reaches it (j <= s_u + kr - kl);
            // window u - 1 reaches it when j < s_u, no earlier one can
            // (kl <= kr).  Both candidates' distances are computed and
            // selected, without a branch; a point in neither measures against
            // p (one broadcast load), the clamped index keeps an empty chunk's
            // loads inside its buffer.  u goes from one of the thread's points
            // to the next (T apart) as quotient and remainder of the
            // non-negative j + kl - p (p <= kl): one division in all.
            const int x0 = c0 + tid + kl - p;
            int u = (int)divq((uint32_t)x0);
            int rem = x0 - u * q;
            const int uT = (int)divq((uint32_t)T);
            const int rT = T - uT * q;
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int jl = tid + T * i;
                const int jlc = max(min(jl, cn - 1), 0);
                const int j = c0 + jlc;  // sector-local index
                const float px = pts[3 * jlc], py = pts[3 * jlc + 1], pz = pts[3 * jlc + 2];
                const int s1 = p + u * q, s0 = s1 - q;
                const bool in1 = jl < cn && u < tw;
                const bool in0 = jl < cn && u >= 1 && u <= tw && j < s1;
                u += uT;  // the quotient of the thread's next point
                rem += rT;
                if (rem >= q) {
                    rem -= q;
                    ++u;
                }
                const int c1 = dev::checked(in1 ? s1 : p, 0, n, a.status);
                const int c0s = dev::checked(in0 ? s0 : p, 0, n, a.status);
                const float d1 = dev::sqdist(px, py, pz, G[3 * c1], G[3 * c1 + 1], G[3 * c1 + 2]);
                const float d0 = dev::sqdist(px, py, pz, G[3 * c0s], G[3 * c0s + 1],
                                             G[3 * c0s + 2]);
                ok = ok && (!in1 || d1 < 1e10f) && (!in0 || d0 < 1e10f);
                float v = D[i];
                v = in1 ? fminf(v, d1) : v;
                v = in0 ? fminf(v, d0) : v;
                D[i] = v;
            }
            bool all = __syncthreads_and(ok) != 0;
            if (CLUSTER) {
                // each CTA's verdict to every peer (buffers alternate between
                // stride phases), one cluster barrier, then every CTA reads all
                const int par = npro & 1;
                if (tid < CS)
                    dev::st_cluster_v4(dev::mapa(dev::smem_u32(&cl_ok[par][rank][0]), (uint32_t)tid),
                                       all ? 1u : 0u, 0u, 0u, 0u);
                dev::cluster_sync();
                for (int r = 0; r < CS; ++r) all = all && cl_ok[par][r][0] != 0u;
                ++npro;
            }
            if (all) {
                if (emitter) {
                    for (int r0 = 0; r0 + 32 <= tn; r0 += 32)
                        out[r0 + lane] = d.lo + p + (r0 + lane) * q;
                    obuf = d.lo + p + (((tn - 1) & ~31) + lane) * q;
                }
                p += (tn - 1) * q;
                qx = G[3 * p];
                qy = G[3 * p + 1];
                qz = G[3 * p + 2];
                t0 = tn;  // re-applying the last window is a no-op
            } else {
#pragma unroll
                for (int i = 0; i < 2 * PP; ++i) D[i] = (i < P && tid + T * i < cn) ? 1e10f : 0.f;
            }
        }

        bool xlate = false;  // the last exchange timed out
        for (int t = t0; t < c; ++t) {
            // 1. update + local argmax (chunk-local offsets)
            const bool whole = full_first && t == 1;  // full first pass reading
            const int wlo = whole ? -c0 : p - kl - c0, whi = whole ? n - 1 - c0 : p + kr - c0;
            const unsigned long long qx2 = dev::pack2(qx, qx), qy2 = dev::pack2(qy, qy),
                                     qz2 = dev::pack2(qz, qz);
            float best = 0.f;
            int bi = 0;
#pragma unroll
            for (int h = 0; h < PP; ++h) {
                const int i0 = 2 * h;
                if (T * i0 < cn || h == 0) {  // CTA-uniform: the row pair holds real points
                    // NPDU: row pairs the window misses are skipped by a CTA-
                    // uniform test (npdu_skip) or computed and masked; inside a
                    // row the window is always a mask, not a branch.
                    const bool hit =
                        !NPDU || !a.npdu_skip || (T * i0 + 2 * T - 1 >= wlo && T * i0 <= whi);
                    if (hit) {
                        // NPDU: a point outside the window takes x = +inf for
                        // this update (distance +inf, D kept); the select
                        // depends on p only, off the critical path.  Padding
                        // holds D = +0, which no update lowers.
                        unsigned long long xh = X2[h];
                        if (NPDU) {
                            const int j0 = tid + T * i0, j1 = j0 + T;
                            const unsigned span = (unsigned)(whi - wlo);
                            float x0, x1;
                            dev::unpack2(xh, x0, x1);
                            x0 = (unsigned)(j0 - wlo) <= span ? x0 : __int_as_float(0x7f800000);
                            x1 = (unsigned)(j1 - wlo) <= span ? x1 : __int_as_float(0x7f800000);
                            xh = dev::pack2(x0, x1);
                        }
                        float d0, d1;
                        dev::sqdist2(xh, Y2[h], Z2[h], qx2, qy2, qz2, d0, d1);
                        D[i0] = fminf(D[i0], d0);
                        D[i0 + 1] = fminf(D[i0 + 1], d1);
                    }
                    if (h == 0) {  // row 0 starts the thread's scan
                        best = D[0];
                        bi = 0;
                    } else {
                        const bool gt = D[i0] > best;  // strict: lowest row wins ties
                        best = gt ? D[i0] : best;
                        bi = gt ? i0 : bi;
                    }
                    if (i0 + 1 < P) {
                        const bool gt = D[i0 + 1] > best;
                        best = gt ? D[i0 + 1] : best;
                        bi = gt ? i0 + 1 : bi;
                    }
                }
            }

            // 2. warp argmax and record
            const unsigned bits = __float_as_uint(best);
            const unsigned m = __reduce_max_sync(dev::kFull, bits);
            const unsigned cand = bits == m ? (unsigned)(tid + T * bi) : 0xffffffffu;
            const unsigned jw = __reduce_min_sync(dev::kFull, cand);  // chunk-local
            const uint32_t jinv = 0xffffffffu - (uint32_t)(c0 + (int)jw);
            const uint32_t xb = xchg & 1u;
            const uint32_t xbar = xb ? xbar1 : xbar0;
            Rec* R = recs + xb * E;
            if (CLUSTER) {
                // The warps' keys meet in this CTA's shared memory; behind one
                // CTA barrier warp 0 reduces them to the CTA's record and its
                // lanes 0..CS-1 send that record, with the winner's x, y, z,
                // to every CTA of the cluster (this one included): CS records
                // per exchange instead of one per warp, so each receiving
                // mbarrier counts CS transfers, not CS x W.
                if (lane == 0) wkeys[w] = make_uint2(m, jinv);
                // a record of the previous exchange that did not come stops
                // the item here (peers stop at their next exchange, which
                // this CTA no longer feeds)
                halted = __syncthreads_or(xlate) != 0;
                if (halted) break;
                if (w == 0) {
                    // every reader of the buffer the previous exchange used has
                    // passed the barrier above: re-arm it before this CTA's
                    // records can let a peer start the next exchange
                    if (lane == 0 && xchg > 0) dev::mbar_arrive_expect_tx(xb ? xbar0 : xbar1, xbytes);
                    const uint2 kv = lane < W ? wkeys[lane] : make_uint2(0u, 0u);
                    const unsigned cm = __reduce_max_sync(dev::kFull, kv.x);
                    const unsigned cj = __reduce_max_sync(dev::kFull, kv.x == cm ? kv.y : 0u);
                    const int jl = dev::checked((int)(0xffffffffu - cj) - c0, 0, T * P, a.status);
                    // fault injection: the cluster's last CTA sends no records
                    const bool send = !((a.stall & STALL_EXCHANGE) && rank == CS - 1);
                    if (lane < CS && send) {
                        const float wx = pts[3 * jl], wy = pts[3 * jl + 1], wz = pts[3 * jl + 2];
                        const uint32_t slot = dev::smem_u32(&R[rank]);
                        const uint32_t remote = dev::mapa(slot, (uint32_t)lane);
                        const uint32_t rbar = dev::mapa(xbar, (uint32_t)lane);
                        dev::st_async_v4(remote, rbar, cm, cj, __float_as_uint(wx),
                                         __float_as_uint(wy));
                        dev::st_async_v4(remote + 16, rbar, __float_as_uint(wz), 0u, 0u, 0u);
                    }
                }
            } else if (lane == 0) {
                *reinterpret_cast<uint2*>(&R[w]) = make_uint2(m, jinv);
            }

            // 3. wait for every record of this exchange
            if (CLUSTER) {
                xlate = !exchange_wait(xbar, xb ? xphase1 : xphase0, a.timeout_ns);
                if (xlate) dev::record_status(a.status, DEV_TIMEOUT_EXCHANGE);
                if (xb)
                    xphase1 ^= 1u;
                else
                    xphase0 ^= 1u;
            } else {
                __syncthreads();
            }

            // 4. every warp reduces the E records: max distance bits, then
            //    the largest ~index (= lowest index) among them
            unsigned long long bkey = 0ull;
            for (int e = lane; e < E; e += 32) {
                const uint2 kv = *reinterpret_cast<const uint2*>(&R[e]);
                const unsigned long long key = ((unsigned long long)kv.x << 32) | kv.y;
                bkey = key > bkey ? key : bkey;
            }
            const unsigned hi = (unsigned)(bkey >> 32), lo = (unsigned)bkey;
            const unsigned mm = __reduce_max_sync(dev::kFull, hi);
            const unsigned lo2 = __reduce_max_sync(dev::kFull, hi == mm ? lo : 0u);
            p = (int)(0xffffffffu - lo2);
            // After a timed-out exchange some records were never written and p
            // may be anything: it is kept inside the sector, so the lookups
            // below stay in bounds, until the CTA stops at its next barrier.
            if (CLUSTER) p = min(max(p, 0), n - 1);
            p = dev::checked(p, 0, n, a.status);
            if (CLUSTER) {
                // the winner's record is its owner CTA's
                const int r = dev::checked((int)dev::SmallDiv((uint32_t)chunk)((uint32_t)p), 0, CS,
                                           a.status);
                qx = R[r].x;
                qy = R[r].y;
                qz = R[r].z;
            } else {
                qx = pts[3 * p];
                qy = pts[3 * p + 1];
                qz = pts[3 * p + 2];
            }
            ++xchg;
            if (emitter) {
                obuf = lane == (t & 31) ? d.lo + p : obuf;
                if ((t & 31) == 31) out[(t & ~31) + lane] = obuf;
            }
        }
        // the item's last exchange timed out: stop here
        if (CLUSTER && !halted) halted = __syncthreads_or(xlate) != 0;
        if (emitter && !halted && lane <= ((c - 1) & 31)) out[((c - 1) & ~31) + lane] = obuf;
    }
    if (CLUSTER) dev::cluster_sync();  // no CTA leaves while a peer may still store to it
}

using SectorKernel = void (*)(LaunchArgs);
SectorKernel warp_kernel_for(int P, bool npdu, bool rows);
SectorKernel win_kernel_for(int rows, bool host_rows, bool lean);
SectorKernel win2_kernel_for(int rows16, bool host_rows);

static SectorKernel cta_kernel_for(int P, bool npdu, bool cluster) {
#define AFPS_CTA_CASE(PP)                                                             \
    case PP:                                                                          \
        if (cluster)                                                                  \
            return npdu ? afps_cta_kernel<PP, true, true> : afps_cta_kernel<PP, false, true>; \
        return npdu ? afps_cta_kernel<PP, true, false> : afps_cta_kernel<PP, false, false>;
    switch (P) {
        AFPS_CTA_CASE(2)
        AFPS_CTA_CASE(4)
        AFPS_CTA_CASE(8)
        AFPS_CTA_CASE(16)
        default:
            return nullptr;
    }
#undef AFPS_CTA_CASE
}

size_t variant_smem(const Variant& v) {
    if (v.kind == KIND_WARP)
        return 16 * ((8 * (size_t)v.W + 15) / 16) + (size_t)v.W * (12 * 32 * (size_t)v.P + 16);
    if (v.kind == KIND_WIN)  // per warp: xyz (12 bytes a point + 16) and distances (4 bytes)
        return 16 * ((8 * (size_t)v.W + 15) / 16) + (size_t)v.W * (16 * 32 * (size_t)v.P + 16);
    if (v.kind == KIND_WIN2)  // two barriers and two such buffers (per half) per warp
        return 16 * (size_t)v.W + 2 * (size_t)v.W * (16 * 16 * (size_t)v.P + 16);
    // records (one per CTA of a cluster, else one per warp), double-buffered;
    // a cluster's CTAs also keep their warps' keys; then the points
    const size_t E = v.CS > 1 ? (size_t)v.CS : (size_t)v.W;
    return 32 + 2 * E * sizeof(Rec) + (v.CS > 1 ? 16 * ((8 * (size_t)v.W + 15) / 16) : 0) +
           12 * 32 * (size_t)v.W * v.P + 16;
}

bool variant_supported(const Variant& v) {
    if (v.kind == KIND_WARP)
        return warp_kernel_for(v.P, false, false) != nullptr && v.W >= 1 && v.W <= 8 && v.CS == 1;
    if (v.kind == KIND_WIN)
        return v.P >= 1 && v.P <= kWinMaxRows && v.W >= 1 && v.W <= 8 && v.CS == 1 &&
               variant_smem(v) <= 227 * 1024;
    if (v.kind == KIND_WIN2)
        return v.P >= 1 && v.P <= kWin2MaxRows && v.W >= 1 && v.W <= 8 && v.CS == 1 &&
               variant_smem(v) <= 227 * 1024;
    if (v.kind != KIND_CTA) return false;
    if (!cta_kernel_for(v.P, false, false)) return false;
    if (v.W < 1 || v.W > (v.P >= 16 ? 8 : 32) || v.CS < 1 || v.CS > 16) return false;
    return variant_smem(v) <= 227 * 1024;
}

// rows: the launch writes its indices to host memory (warp kernels then
// store them as rows of 32)
static SectorKernel kernel_for(const Variant& v, bool npdu, bool rows = false) {
    if (v.kind == KIND_WARP) return warp_kernel_for(v.P, npdu, rows);
    if (v.kind == KIND_WIN) return win_kernel_for(v.P, rows, v.skip != 0);
    if (v.kind == KIND_WIN2) return win2_kernel_for(v.P, rows);
    return cta_kernel_for(v.P, npdu, v.CS > 1);
}

// Function attributes for a launch, set only when they must grow: the
// dynamic shared-memory attribute is an upper bound, so each (device,
// kernel) keeps the largest value set so far, and the non-portable cluster
// permission is set once.  Setting them on every launch costs host time.
static cudaError_t prepare(SectorKernel fn, const Variant& v, size_t smem) {
    static std::mutex mu;
    static std::map<std::pair<int, const void*>, size_t> smem_set;
    static std::set<std::pair<int, const void*>> wide_set;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const void* f = reinterpret_cast<const void*>(fn);
    const auto key = std::make_pair(dev, f);
    const bool wide = v.kind == KIND_CTA && v.CS > 8;
    std::lock_guard<std::mutex> lock(mu);
    auto it = smem_set.find(key);
    if (it == smem_set.end() || it->second < smem) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        smem_set[key] = smem;
    }
    if (wide && !wide_set.count(key)) {
        e = cudaFuncSetAttribute(f, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
        wide_set.insert(key);
    }
    return cudaSuccess;
}

cudaError_t launch_sector(const Variant& v, bool npdu, const LaunchArgs& args, int grid,
                          cudaStream_t stream) {
    if (!variant_supported(v) || grid < 1) return cudaErrorInvalidValue;
    if ((v.kind == KIND_WIN || v.kind == KIND_WIN2) && !npdu)
        return cudaErrorInvalidValue;  // windows only
    LaunchArgs a = args;
    a.win_cap = v.kind == KIND_WIN ? 32 * v.P : v.kind == KIND_WIN2 ? 16 * v.P : 0;
    SectorKernel fn = kernel_for(v, npdu, a.host_resident != 0);
    const size_t smem = variant_smem(v);
    cudaError_t e = prepare(fn, v, smem);
    if (e != cudaSuccess) return e;
    if (v.kind == KIND_CTA && v.CS > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)(grid * v.CS), 1, 1);
        cfg.blockDim = dim3((unsigned)(32 * v.W), 1, 1);
        cfg.dynamicSmemBytes = smem;
        cfg.stream = stream;
        cudaLaunchAttribute attr[2];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)v.CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        attr[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[1].val.programmaticStreamSerializationAllowed = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 2;
        return cudaLaunchKernelEx(&cfg, fn, a);
    }
    // Programmatic dependent launch: the kernels wait (griddepcontrol.wait)
    // before touching global memory, so they may be scheduled while the
    // previous kernel of the stream is still running.
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3((unsigned)(32 * v.W), 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, fn, a);
}

int max_active_clusters(const Variant& v) {
    if (!variant_supported(v)) return 0;
    SectorKernel fn = kernel_for(v, false);
    const size_t smem = variant_smem(v);
    if (prepare(fn, v, smem) != cudaSuccess) return 0;
    if (v.kind == KIND_CTA && v.CS > 1) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)v.CS, 1, 1);
        cfg.blockDim = dim3((unsigned)(32 * v.W), 1, 1);
        cfg.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)v.CS;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int n = 0;
        if (cudaOccupancyMaxActiveClusters(&n, fn, &cfg) != cudaSuccess) return 0;
        return n;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, 32 * v.W, smem) !=
        cudaSuccess)
        return 0;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return per_sm * sms;
}

}  // namespace afps
