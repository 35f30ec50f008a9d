// afps_warp.cu -- one warp per sector (Sec. III-B), for sectors of up to
// 32 * P points.
//
// Each warp owns one (cloud, sector) work item at a time:
//   stage-in   the sector's xyz (12 bytes per point, contiguous in storage
//              order) goes HBM -> shared memory by one bulk copy on the TMA
//              engine (16-byte aligned interior) plus plain loads of the
//              unaligned head and tail; lane l then keeps points l + 32 i
//              (i < P) in registers, with their running distance (1e10,
//              Algorithm 1).  Shared memory keeps the xyz for looking up the
//              coordinates of each new sample.
//   iteration  distance update of the points the new sample reaches (all of
//              the sector, or the NPDU window of Sec. III-C), fused with each
//              lane's local argmax; then the warp argmax as two redux.sync
//              steps: max of the distance bits (distances are >= +0, so the
//              unsigned bit order is the float order), then min of the index
//              among the lanes holding that maximum (lowest index on ties).
//   emit       every lane learns each sample from the reduction; lane 0
//              stores it (the stride phase's samples go out as coalesced
//              rows); indices in host memory go out as rows of 32.
// Work items come from a device counter (dynamic queue) or by static
// striding.  No CTA-wide synchronisation: warps of a CTA are independent.
#include "afps_device.cuh"

namespace afps {

// ROWS: the indices go to host memory (over the C2C link), as rows of 32.
template <int P, bool NPDU, bool ROWS>
__global__ void __launch_bounds__(256) afps_warp_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int kBuf = 12 * 32 * P + 16;
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* buf = smem + 16 * ((8 * W + 15) / 16) + w * kBuf;
    const uint32_t bar = dev::smem_u32(&bars[w]);
    if (lane == 0) {
        dev::mbar_init(bar, 1);
        dev::fence_mbar_init();
    }
    __syncwarp();
    // A computed first item (no table, no cloud records, no queue) needs no
    // memory access, so its points can be prefetched into L2 while the
    // previous kernel of the stream still runs.
    if (!a.items && !a.single.clouds && !a.counter && !a.host_resident &&
        blockIdx.x * W + w < a.n_items) {
        const ItemDesc d0 = dev::load_item(a, blockIdx.x * W + w);
        const char* g = reinterpret_cast<const char*>(a.xyz + 3 * d0.src);
        for (int off = 128 * lane; off < 12 * d0.n; off += 32 * 128) dev::prefetch_l2(g + off);
    }
    // Programmatic dependent launch: wait until the previous kernel of the
    // stream has completed (no global memory access before this), then let
    // the next one be scheduled: one kernel waits behind a running one, and
    // the chain never grows deeper than that.
    dev::pdl_wait();
    dev::pdl_launch_dependents();
    uint32_t phase = 0;
    bool halted = false;  // a timeout was seen: leave the remaining items undone

    const int nwarps = gridDim.x * W;
    int item = a.counter ? dev::queue_next(a, nwarps, lane) : blockIdx.x * W + w;

    for (; item < a.n_items;
         item = a.counter ? dev::queue_next(a, nwarps, lane) : item + nwarps) {
        if (halted) continue;
        const ItemDesc d = dev::load_item(a, item);
        const int n = dev::checked(d.n, 1, 32 * P + 1, a.status);  // fits the staging buffer

        // ---- stage-in (the previous item's readers are done: fence + sync)
        dev::fence_proxy_async_smem();
        __syncwarp();
        bool bulk;
        const float* pts =
            dev::stage_points(a.xyz + 3 * d.src, n, buf, bar, lane == 0, lane, 32, &bulk,
                              (a.stall & STALL_COPY) != 0, a.host_resident != 0);
        // a timeout recorded by any warp so far (the load overlaps the copy)
        const int seen = dev::load_status(a.status);
        bool late = false;
        if (bulk) {
            late = !dev::mbar_wait_bounded(bar, phase, a.timeout_ns);
            if (late) {
                dev::record_status(a.status, DEV_TIMEOUT_STAGE);
                if (!dev::mbar_wait_bounded(bar, phase, a.timeout_ns))
                    dev::record_status(a.status, DEV_TIMEOUT_DRAIN);
            }
            phase ^= 1u;
        }
        __syncwarp();
        // after a timeout (here or anywhere on the context) nothing is
        // computed on shared memory the copy may not have filled; the warp
        // only draws its remaining tickets
        halted = __any_sync(dev::kFull, late || dev::is_timeout(seen));
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
                const int j = lane + 32 * i;
                if (i < P && j < n) {
                    xs[u] = pts[3 * j];
                    ys[u] = pts[3 * j + 1];
                    zs[u] = pts[3 * j + 2];
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

        int32_t* out = a.out + d.dst;
        const int c = dev::checked(d.c, 1, n + 1, a.status);
        const int kl = d.kl;
        const int kr = d.kr;
        const bool full_first = (d.flags & ITEM_FULL_FIRST) != 0;
        int p = dev::checked(d.first, 0, n, a.status);
        // Every lane knows each sample.  Indices in device memory: lane 0
        // stores each one (one instruction per sample; buffering them for
        // row stores costs a select per sample).  Indices in host memory,
        // written over the C2C link, where each store is a transfer: lane t
        // % 32 keeps sample t and the warp stores full rows of 32.
        constexpr bool rows_out = ROWS;
        int obuf = lane == 0 ? d.lo + p : 0;
        if (lane == 0 && !rows_out) out[0] = d.lo + p;
        int t0 = 1;
        if (NPDU && !full_first && p <= kl && kl <= kr) {
            // Stride phase of the literal NPDU reading (distances start at
            // 1e10, Sec. III-C): while points past the last window are
            // untouched they hold the maximum 1e10, so the lowest-index argmax
            // is the first of them and the samples are p, p + q, p + 2q, ...
            // (q = kr + 1) until a window reaches the sector's end.  Their
            // window updates are independent and run here at once; the argmax
            // scans they replace are decided in advance, provided every
            // windowed distance is below 1e10 (else the serial loop runs from
            // the start).  With kl <= kr a point lies in at most two windows.
            const int q = kr + 1;
            const int x = n - 1 - kr - p;
            const dev::SmallDiv divq((uint32_t)q);
            const int ts = x <= 0 ? 1 : (int)divq((uint32_t)(x + q - 1)) + 1;  // stride length
            const int tn = min(ts, c);                        // of them emitted
            const int tw = min(ts, c - 1);                    // whose window is applied
            bool ok = true;  // D is updated in place and reset if the test fails
            // Window u = floor((j + kl - p) / q) is the last one starting at or
            // before point j (p <= kl, so the quotient is of a non-negative
            // number); window u - 1 may reach j too, no earlier one can
            // (kl <= kr).  Both candidates' distances are computed from
            // clamped indices and selected: no branch, one division a point.
#pragma unroll
            for (int i = 0; i < P; ++i) {
                const int j = lane + 32 * i;
                const int jc = min(j, n - 1);
                const float px = pts[3 * jc], py = pts[3 * jc + 1], pz = pts[3 * jc + 2];
                const int u = (int)divq((uint32_t)(jc + kl - p));
                const int s1 = p + u * q, s0 = s1 - q;
                const bool in1 = j < n && u < tw && jc <= s1 + kr;
                const bool in0 = j < n && u >= 1 && u - 1 < tw && jc < s1;
                const int c1 = dev::checked(in1 ? s1 : jc, 0, n, a.status);
                const int c0 = dev::checked(in0 ? s0 : jc, 0, n, a.status);
                const float d1 = dev::sqdist(px, py, pz, pts[3 * c1], pts[3 * c1 + 1],
                                             pts[3 * c1 + 2]);
                const float d0 = dev::sqdist(px, py, pz, pts[3 * c0], pts[3 * c0 + 1],
                                             pts[3 * c0 + 2]);
                ok = ok && (!in1 || d1 < 1e10f) && (!in0 || d0 < 1e10f);
                float v = D[i];
                v = in1 ? fminf(v, d1) : v;
                v = in0 ? fminf(v, d0) : v;
                D[i] = v;
            }
            if (__all_sync(dev::kFull, ok)) {
                if (rows_out) {
                    for (int r0 = 0; r0 + 32 <= tn; r0 += 32) out[r0 + lane] = d.lo + p + (r0 + lane) * q;
                    obuf = d.lo + p + (((tn - 1) & ~31) + lane) * q;
                } else {
                    for (int t = 1 + lane; t < tn; t += 32) out[t] = d.lo + p + t * q;
                }
                p += (tn - 1) * q;
                t0 = tn;  // re-applying the last window is a no-op
            } else {
#pragma unroll
                for (int i = 0; i < 2 * PP; ++i) D[i] = (i < P && lane + 32 * i < n) ? 1e10f : 0.f;
            }
        }
        // One argmax round: the update by the last sample p of the points in
        // [wl, wh] (its NPDU window, or the whole sector), fused with each
        // lane's argmax over its rows, then the warp argmax as two redux.sync
        // steps (max of the distance bits, min of the index among the lanes
        // holding it); stores sample t.
        auto round = [&](int t, int wl, int wh) {
            const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
            const unsigned long long qx2 = dev::pack2(qx, qx), qy2 = dev::pack2(qy, qy),
                                     qz2 = dev::pack2(qz, qz);
            const unsigned wlo = (unsigned)wl;  // [wl, wh] as one unsigned range test
            const unsigned wspan = (unsigned)(wh - wl);
            float best = 0.f;
            int bi = 0;
#pragma unroll
            for (int h = 0; h < PP; ++h) {
                const int i0 = 2 * h;
                if (h == 0 || 32 * i0 < n) {  // warp-uniform: the row pair holds real points (n >= 1)
                    // NPDU: every row pair is computed and the window applied as
                    // a mask, or (npdu_skip) pairs the window misses are skipped
                    // by a warp-uniform test; never a divergent branch.  With
                    // one pair the window always reaches it.
                    const bool hit = !NPDU || PP == 1 || !a.npdu_skip ||
                                     (32 * i0 + 63 >= wl && 32 * i0 <= wh);
                    if (hit) {
                        // NPDU: a point outside the window takes x = +inf for
                        // this update, so its distance is +inf and the min
                        // keeps D; inside, the arithmetic is unchanged.  The
                        // select depends only on p, not on the sample's
                        // coordinates, so it stays off the round's critical
                        // path.  (Padding holds D = +0, which no update lowers.)
                        unsigned long long xh = X2[h];
                        if (NPDU) {
                            const int j0 = lane + 32 * i0, j1 = j0 + 32;
                            float x0, x1;
                            dev::unpack2(xh, x0, x1);
                            x0 = ((unsigned)j0 - wlo) <= wspan ? x0 : __int_as_float(0x7f800000);
                            x1 = ((unsigned)j1 - wlo) <= wspan ? x1 : __int_as_float(0x7f800000);
                            xh = dev::pack2(x0, x1);
                        }
                        float d0, d1;
                        dev::sqdist2(xh, Y2[h], Z2[h], qx2, qy2, qz2, d0, d1);
                        D[i0] = fminf(D[i0], d0);
                        D[i0 + 1] = fminf(D[i0 + 1], d1);
                    }
                    if (h == 0) {  // row 0 starts the lane's scan
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
            const unsigned bits = __float_as_uint(best);
            const unsigned m = __reduce_max_sync(dev::kFull, bits);
            const unsigned cand = bits == m ? (unsigned)(lane + 32 * bi) : 0xffffffffu;
            p = dev::checked((int)__reduce_min_sync(dev::kFull, cand), 0, n, a.status);
            if (rows_out) {
                obuf = lane == (t & 31) ? d.lo + p : obuf;
                if ((t & 31) == 31) out[(t & ~31) + lane] = obuf;
            } else if (lane == 0) {
                out[t] = d.lo + p;
            }
        };
        int t = t0;
        if (full_first && t < c) round(t++, 0, n - 1);  // full-first-pass reading: the first update is the whole sector
        // small rounds unrolled: the loop's own instructions are a fair share of them
#pragma unroll(P <= 4 ? 4 : 1)
        for (; t < c; ++t) round(t, p - kl, p + kr);
        if (rows_out && lane <= ((c - 1) & 31)) out[((c - 1) & ~31) + lane] = obuf;
    }
}

using SectorKernel = void (*)(LaunchArgs);

SectorKernel warp_kernel_for(int P, bool npdu, bool rows) {
#define AFPS_WARP_CASE(PP)                                                              \
    case PP:                                                                            \
        if (rows) return npdu ? afps_warp_kernel<PP, true, true> : afps_warp_kernel<PP, false, true>; \
        return npdu ? afps_warp_kernel<PP, true, false> : afps_warp_kernel<PP, false, false>;
    switch (P) {
        AFPS_WARP_CASE(1)
        AFPS_WARP_CASE(2)
        AFPS_WARP_CASE(3)
        AFPS_WARP_CASE(4)
        AFPS_WARP_CASE(6)
        AFPS_WARP_CASE(8)
        AFPS_WARP_CASE(12)
        AFPS_WARP_CASE(16)
        AFPS_WARP_CASE(24)
        AFPS_WARP_CASE(32)
        default:
            return nullptr;
    }
#undef AFPS_WARP_CASE
}

}  // namespace afps
