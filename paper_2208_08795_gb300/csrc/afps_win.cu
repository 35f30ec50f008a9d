// afps_win.cu -- NPDU sectors (Sec. III-C) at a constant cost per iteration.
//
// One warp per (cloud, sector) work item, sectors of up to 32 * 32 * R points.
// The register kernels (afps_warp.cu, afps_cta.cu) rescan every running
// distance of the sector for each argmax, although NPDU changes only the k + 1
// distances of the window.  Here the distances live in shared memory beside
// the staged xyz, and the warp caches the maximum of each row of 32 points
// (lane l holds the maxima of rows l, l + 32, ...: R slots).  An iteration
// touches only what its window touches:
//   update   lane i updates point wl + i of the window [wl, wh] (the k
//            neighbours and the sample, clipped to the sector) in shared
//            memory: d = (dx*dx + dy*dy) + dz*dz, D = min(D, d);
//   rows     every row the window overlaps (at most two for k < 32) gets its
//            maximum recomputed: redux.sync max of the distance bits, then
//            redux.sync min of the lane among those that hold it;
//   argmax   each lane offers the best of its cached rows that the window
//            missed and of its own column of the touched rows; two redux.sync
//            steps give the maximum and the lowest index that holds it.
// Distances only decrease, so a row the window misses keeps its maximum and
// the lowest index attaining it: the result is exactly the lowest-index
// argmax of a full scan (Algorithm 1), bit for bit.
//
// The stride phase of the literal reading (every distance starts at 1e10, no
// first full pass; the first samples are p, p + q, p + 2q, ... while points
// past the last window are untouched) runs as one parallel pass, as in the
// register kernels, and computes every row maximum on the way.
#include "afps_device.cuh"

namespace afps {

namespace {

// Row r's maximum (distance bits m, index idx) into the slot of its owner
// lane r % 32 (slot r / 32).
template <int R>
__device__ __forceinline__ void set_row(unsigned (&rmb)[R], unsigned (&rmi)[R], int r,
                                        unsigned m, unsigned idx, int lane, int lanes = 32) {
#pragma unroll
    for (int s = 0; s < R; ++s)
        if (r == lane + lanes * s) {
            rmb[s] = m;
            rmi[s] = idx;
        }
}

// Every row's maximum is 1e10 at its first point; a slot past the last row
// holds +0 at no index and loses every tie.
template <int R>
__device__ __forceinline__ void reset_slots(int rows, unsigned (&rmb)[R], unsigned (&rmi)[R],
                                            int lane) {
#pragma unroll
    for (int s = 0; s < R; ++s) {
        const int r = lane + 32 * s;
        rmb[s] = r < rows ? __float_as_uint(1e10f) : 0u;
        rmi[s] = r < rows ? (unsigned)(32 * r) : 0xffffffffu;
    }
}

// Every distance at 1e10 (points) or +0 (the padding of the last row, which
// loses every tie).
__device__ __forceinline__ void reset_dist(float* Ds, int n, int rows, int lane) {
    for (int j = lane; j < 32 * rows; j += 32) Ds[j] = j < n ? 1e10f : 0.f;
}

// The lowest-index maximum of row r from its 32 distance bits (one per lane).
__device__ __forceinline__ void row_max(unsigned b, int lane, unsigned& m, unsigned& l) {
    m = __reduce_max_sync(dev::kFull, b);
    l = __reduce_min_sync(dev::kFull, b == m ? (unsigned)lane : 32u);
}

}  // namespace

// ROWS: the indices go to host memory (over the C2C link), as rows of 32.
// LEAN: the narrow round with the fewest instructions (the touched rows'
// cache entries first, then the argmax over the cache) instead of the one
// with the shortest dependency chain; the autotuner picks per shape class.
template <int R, bool ROWS, bool LEAN>
__global__ void __launch_bounds__(256) afps_win_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int w = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int cap = a.win_cap;  // points per warp: xyz 12 cap + 16 bytes, distances 4 cap
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);
    unsigned char* buf = smem + 16 * ((8 * W + 15) / 16) + (size_t)w * (16 * (size_t)cap + 16);
    float* Ds = reinterpret_cast<float*>(buf + 12 * (size_t)cap + 16);
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
    // Programmatic dependent launch, as in the other sector kernels.
    dev::pdl_wait();
    dev::pdl_launch_dependents();
    uint32_t phase = 0;
    bool halted = false;  // a timeout was seen: leave the remaining items undone

    const int nwarps = gridDim.x * W;
    int item = a.counter ? dev::queue_next(a, nwarps, lane) : blockIdx.x * W + w;

    while (item < a.n_items) {
        if (!halted) {
            const ItemDesc d = dev::load_item(a, item);
            const int n = dev::checked(d.n, 1, cap + 1, a.status);  // fits the warp's buffer

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
            halted = __any_sync(dev::kFull, late || dev::is_timeout(seen));
            if (!halted) {
                const int rows = (n + 31) >> 5;
                unsigned rmb[R], rmi[R];  // cached row maxima: bits, lowest index
                reset_slots<R>(rows, rmb, rmi, lane);
                int32_t* out = a.out + d.dst;
                const int c = dev::checked(d.c, 1, n + 1, a.status);
                const int kl = d.kl;
                const int kr = d.kr;
                const bool full_first = (d.flags & ITEM_FULL_FIRST) != 0;
                int p = dev::checked(d.first, 0, n, a.status);
                // Device indices: lane 0 stores each sample.  Host indices (C2C
                // link, where each store is a transfer): lane t % 32 keeps
                // sample t and the warp stores rows of 32.
                int obuf = lane == 0 ? d.lo + p : 0;
                if (lane == 0 && !ROWS) out[0] = d.lo + p;
                int t0 = 1;
                bool fresh = true;  // distances still to be set to 1e10
                if (!full_first && p <= kl && kl <= kr) {
                    // Stride phase (see afps_warp.cu): samples p, p + q, ...
                    // (q = kr + 1) until a window reaches the sector's end;
                    // their windows are applied at once, valid if every
                    // windowed distance is below 1e10.  Point j lies in window
                    // u = floor((j + kl - p) / q) (the last one starting at or
                    // before it, which always reaches it since kl <= kr) and
                    // possibly in window u - 1.  Every distance, padding
                    // included, is written here, and rows are visited in
                    // order, so each row's maximum comes from registers.
                    const int q = kr + 1;
                    const int x = n - 1 - kr - p;
                    const dev::SmallDiv divq((uint32_t)q);
                    const int ts = x <= 0 ? 1 : (int)divq((uint32_t)(x + q - 1)) + 1;
                    const int tn = min(ts, c);      // stride samples emitted
                    const int tw = min(ts, c - 1);  // ... whose window is applied
                    bool ok = true;
                    // u = floor((j + kl - p) / q) for j = 32 i + lane (a
                    // non-negative numerator: p <= kl), carried from row to
                    // row as quotient and remainder instead of one division
                    // a point.  Window u always reaches j (j <= s_u + kr - kl);
                    // window u - 1 reaches it when j < s_u (its last point is
                    // s_u - q + kr = s_u - 1).
                    const int x0 = lane + kl - p;
                    int u = (int)divq((uint32_t)x0);
                    int rem = x0 - u * q;
                    const int u32 = (int)divq(32u);
                    const int r32 = 32 - u32 * q;
                    for (int i = 0; i < rows; ++i) {
                        const int j = 32 * i + lane;
                        // both candidate windows' distances are computed (from a
                        // clamped point) and selected, without a branch
                        const int jc = min(j, n - 1);
                        const float px = pts[3 * jc], py = pts[3 * jc + 1], pz = pts[3 * jc + 2];
                        const int s1 = p + u * q, s0 = s1 - q;  // windows u and u - 1
                        const bool in1 = j < n && u < tw;
                        const bool in0 = j < n && u >= 1 && u <= tw && j < s1;
                        u += u32;  // the next row's quotient
                        rem += r32;
                        if (rem >= q) {
                            rem -= q;
                            ++u;
                        }
                        const int c1 = dev::checked(in1 ? s1 : jc, 0, n, a.status);
                        const int c0 = dev::checked(in0 ? s0 : jc, 0, n, a.status);
                        const float d1 = dev::sqdist(px, py, pz, pts[3 * c1], pts[3 * c1 + 1],
                                                     pts[3 * c1 + 2]);
                        const float d0 = dev::sqdist(px, py, pz, pts[3 * c0], pts[3 * c0 + 1],
                                                     pts[3 * c0 + 2]);
                        ok = ok && (!in1 || d1 < 1e10f) && (!in0 || d0 < 1e10f);
                        float v = j < n ? 1e10f : 0.f;  // padding: +0
                        v = in1 ? fminf(v, d1) : v;
                        v = in0 ? fminf(v, d0) : v;
                        Ds[j] = v;
                        unsigned m, l;
                        row_max(__float_as_uint(v), lane, m, l);
                        set_row<R>(rmb, rmi, i, m, (unsigned)(32 * i) + l, lane);
                    }
                    fresh = false;
                    if (__all_sync(dev::kFull, ok)) {
                        if (ROWS) {
                            for (int r0 = 0; r0 + 32 <= tn; r0 += 32)
                                out[r0 + lane] = d.lo + p + (r0 + lane) * q;
                            obuf = d.lo + p + (((tn - 1) & ~31) + lane) * q;
                        } else {
                            for (int t = 1 + lane; t < tn; t += 32) out[t] = d.lo + p + t * q;
                        }
                        p += (tn - 1) * q;
                        t0 = tn;  // re-applying the last window is a no-op
                    } else {
                        fresh = true;
                        reset_slots<R>(rows, rmb, rmi, lane);
                    }
                }
                if (fresh) {
                    __syncwarp();
                    reset_dist(Ds, n, rows, lane);
                }
                __syncwarp();

                // General round: the window [wl, wh] of the last sample p (the
                // whole sector for the first update of the full-first-pass
                // reading, or a window wider than a row): one lane per point,
                // every touched row's maximum recomputed.
                auto round_any = [&](int t, int wl, int wh) {
                    const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
                    for (int j = wl + lane; j <= wh; j += 32) {
                        const float dd =
                            dev::sqdist(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2], qx, qy, qz);
                        Ds[j] = fminf(Ds[j], dd);
                    }
                    __syncwarp();
                    const int r0 = wl >> 5, r1 = wh >> 5;
                    // this lane's candidate: its cached rows the window missed ...
                    unsigned cb = 0u, ci = 0xffffffffu;
#pragma unroll
                    for (int s = 0; s < R; ++s) {
                        const int r = lane + 32 * s;
                        const bool kept = r < r0 || r > r1;
                        const bool better = rmb[s] > cb || (rmb[s] == cb && rmi[s] < ci);
                        cb = kept && better ? rmb[s] : cb;
                        ci = kept && better ? rmi[s] : ci;
                    }
                    // ... and its column of the rows it touched, whose maxima
                    // are recomputed
                    for (int r = r0; r <= r1; ++r) {
                        const unsigned j = (unsigned)(32 * r + lane);
                        const unsigned b = __float_as_uint(Ds[j]);
                        const bool better = b > cb || (b == cb && j < ci);
                        cb = better ? b : cb;
                        ci = better ? j : ci;
                        unsigned m, l;
                        row_max(b, lane, m, l);
                        set_row<R>(rmb, rmi, r, m, (unsigned)(32 * r) + l, lane);
                    }
                    const unsigned mx = __reduce_max_sync(dev::kFull, cb);
                    p = dev::checked((int)__reduce_min_sync(dev::kFull, cb == mx ? ci : 0xffffffffu),
                                     0, n, a.status);
                    if (ROWS) {
                        obuf = lane == (t & 31) ? d.lo + p : obuf;
                        if ((t & 31) == 31) out[(t & ~31) + lane] = obuf;
                    } else if (lane == 0) {
                        out[t] = d.lo + p;
                    }
                };
                int t = t0;
                if (full_first && t < c) round_any(t++, 0, n - 1);
                if (LEAN && kl + kr <= 31) {
                    // Narrow window, fewest instructions: the touched rows' cache
                    // entries are recomputed first (the sample's row, and the
                    // other row the window crosses into only when its cached
                    // maximum lies in the window), then the sample is the argmax over
                    // the cache: every lane's best slot (slots ascend, so the
                    // first of equal maxima has the lowest index), two redux.sync
                    // steps.  One row: four redux.sync, two rows: six.  Unrolled
                    // four times: 63 warp instructions per round instead of 69.5.
                    const int nm1 = n - 1;
#pragma unroll 4
                    for (; t < c; ++t) {
                        const int wl = max(p - kl, 0);
                        const int wh = min(p + kr, nm1);
                        const int j = min(wl + lane, wh);  // past the end: the last point again
                        const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
                        const float dd = dev::sqdist(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2],
                                                     qx, qy, qz);
                        Ds[j] = fminf(Ds[j], dd);
                        __syncwarp();
                        const int r0 = wl >> 5, r1 = wh >> 5;
                        const int rp = p >> 5;  // the sample's row
                        {
                            const unsigned b0 = __float_as_uint(Ds[32 * rp + lane]);
                            unsigned m0, l0;
                            row_max(b0, lane, m0, l0);
                            set_row<R>(rmb, rmi, rp, m0, (unsigned)(32 * rp) + l0, lane);
                        }
                        if (r1 != r0) {
                            // The other touched row keeps its cached maximum and
                            // index unless that index lies in the window (its
                            // points only decreased); a warp-uniform test on the
                            // entry, fetched from its owner lane.
                            const int ro = r0 + r1 - rp;
                            unsigned v = rmi[0];
#pragma unroll
                            for (int s = 1; s < R; ++s) v = (ro >> 5) == s ? rmi[s] : v;
                            const unsigned io = __shfl_sync(dev::kFull, v, ro & 31);
                            if (io - (unsigned)wl <= (unsigned)(wh - wl)) {
                                const unsigned b1 = __float_as_uint(Ds[32 * ro + lane]);
                                unsigned m1, l1;
                                row_max(b1, lane, m1, l1);
                                set_row<R>(rmb, rmi, ro, m1, (unsigned)(32 * ro) + l1, lane);
                            }
                        }
                        unsigned cb = rmb[0], ci = rmi[0];
#pragma unroll
                        for (int s = 1; s < R; ++s) {
                            const bool gt = rmb[s] > cb;
                            cb = gt ? rmb[s] : cb;
                            ci = gt ? rmi[s] : ci;
                        }
                        const unsigned mx = __reduce_max_sync(dev::kFull, cb);
                        p = dev::checked((int)__reduce_min_sync(dev::kFull, cb == mx ? ci : 0xffffffffu),
                                         0, n, a.status);
                        if (ROWS) {
                            obuf = lane == (t & 31) ? d.lo + p : obuf;
                            if ((t & 31) == 31) out[(t & ~31) + lane] = obuf;
                        } else if (lane == 0) {
                            out[t] = d.lo + p;
                        }
                    }
                } else if (kl + kr <= 31) {
                    // Narrow window (at most 32 points): lane i updates point
                    // wl + i; the window touches row r0 and perhaps r1 = r0 + 1.
                    // The maxima of the touched rows (m0, m1) and of the cached
                    // rows it missed (mk) are reduced side by side; the sample is
                    // the lowest index holding the largest of the three.  The
                    // touched rows' lowest-index lanes, needed only by the next
                    // rounds' cache, come after it.
                    const int nm1 = n - 1;
#pragma unroll 4
                    for (; t < c; ++t) {
                        const int wl = max(p - kl, 0);
                        const int wh = min(p + kr, nm1);
                        // lanes past the window's end all update its last point
                        // with the same value: no branch, no divergence
                        const int j = min(wl + lane, wh);
                        const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
                        const float dd = dev::sqdist(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2],
                                                     qx, qy, qz);
                        Ds[j] = fminf(Ds[j], dd);
                        __syncwarp();
                        const int r0 = wl >> 5, r1 = wh >> 5;
                        const unsigned j0 = (unsigned)(32 * r0 + lane);
                        const unsigned j1 = (unsigned)(32 * r1 + lane);
                        const unsigned b0 = __float_as_uint(Ds[j0]);
                        const unsigned b1 = __float_as_uint(Ds[j1]);  // = b0 with one row
                        unsigned kb = 0u, ki = 0xffffffffu;  // best cached row it missed
#pragma unroll
                        for (int s = 0; s < R; ++s) {
                            const int r = lane + 32 * s;
                            const bool take = r != r0 && r != r1 && (rmb[s] > kb || ki == 0xffffffffu);
                            kb = take ? rmb[s] : kb;
                            ki = take ? rmi[s] : ki;
                        }
                        const unsigned m0 = __reduce_max_sync(dev::kFull, b0);
                        const unsigned m1 = __reduce_max_sync(dev::kFull, b1);
                        const unsigned mk = __reduce_max_sync(dev::kFull, kb);
                        const unsigned mx = max(max(m0, m1), mk);
                        unsigned cand = b1 == mx ? j1 : 0xffffffffu;
                        cand = b0 == mx ? j0 : cand;
                        cand = kb == mx && ki < cand ? ki : cand;
                        p = dev::checked((int)__reduce_min_sync(dev::kFull, cand), 0, n, a.status);
                        const unsigned l0 = __reduce_min_sync(dev::kFull, b0 == m0 ? (unsigned)lane : 32u);
                        set_row<R>(rmb, rmi, r0, m0, (unsigned)(32 * r0) + l0, lane);
                        if (r1 != r0) {
                            const unsigned l1 =
                                __reduce_min_sync(dev::kFull, b1 == m1 ? (unsigned)lane : 32u);
                            set_row<R>(rmb, rmi, r1, m1, (unsigned)(32 * r1) + l1, lane);
                        }
                        if (ROWS) {
                            obuf = lane == (t & 31) ? d.lo + p : obuf;
                            if ((t & 31) == 31) out[(t & ~31) + lane] = obuf;
                        } else if (lane == 0) {
                            out[t] = d.lo + p;
                        }
                    }
                } else {
#pragma unroll 1
                    for (; t < c; ++t) round_any(t, max(p - kl, 0), min(p + kr, n - 1));
                }
                if (ROWS && lane <= ((c - 1) & 31)) out[((c - 1) & ~31) + lane] = obuf;
            }
        }
        item = a.counter ? dev::queue_next(a, nwarps, lane) : item + nwarps;
    }
}

// ---------------------------------------------------------------- pairs
// Two sectors per warp, one per half-warp of 16 lanes, for windows of at most
// 17 points (kl + kr <= 16) read literally (no full first pass).  A round's
// bookkeeping (window bounds, the touched rows, the reductions, the store)
// is then shared by two sectors: every instruction serves both halves, each
// with its own data; a reduction takes two full-warp redux.sync steps (one
// per half) or one ballot.  The sample's own distance becomes +0 without arithmetic
// (its distance to itself is exactly +0), so its 16 neighbours take one lane
// each.  Rows are 16 points; half-lane h caches rows h, h + 16, ... (R
// slots, sectors of up to 256 R points).  Rounds take the lean form (the
// touched rows' cache entries, then the argmax over the cache), and the two
// halves run them in lockstep: the loop runs while either half has rounds
// left, a half past its last round computes without storing, and both rows
// a window may touch are reduced every round (the second is the first again
// when the window stays in one row), so no branch splits the warp.
// Per-half reductions with the full warp's mask: the other half's lanes
// contribute the operation's identity, and each lane keeps its own half's
// result.  (Each half naming only its own 16 lanes would give two different
// member masks in one instruction.)
__device__ __forceinline__ unsigned half_max(unsigned v, int half) {
    const unsigned lo = __reduce_max_sync(dev::kFull, half ? 0u : v);
    const unsigned hi = __reduce_max_sync(dev::kFull, half ? v : 0u);
    return half ? hi : lo;
}
__device__ __forceinline__ unsigned half_min(unsigned v, int half) {
    const unsigned lo = __reduce_min_sync(dev::kFull, half ? 0xffffffffu : v);
    const unsigned hi = __reduce_min_sync(dev::kFull, half ? v : 0xffffffffu);
    return half ? hi : lo;
}
// Lowest lane of this half (0..15) where pred holds; pred must hold somewhere.
__device__ __forceinline__ unsigned half_first(bool pred, unsigned hmask, int half) {
    return (unsigned)(__ffs((int)(__ballot_sync(dev::kFull, pred) & hmask)) - 1 - 16 * half);
}

template <int R, bool ROWS>
__global__ void __launch_bounds__(256) afps_win2_kernel(const LaunchArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int lane = threadIdx.x & 31;
    const int half = lane >> 4, hl = lane & 15;
    const unsigned hmask = half ? 0xffff0000u : 0x0000ffffu;
    const int w = threadIdx.x >> 5;
    const int W = blockDim.x >> 5;
    const int cap = a.win_cap;  // points per half buffer: xyz 12 cap + 16 bytes, distances 4 cap
    uint64_t* bars = reinterpret_cast<uint64_t*>(smem);  // two per warp
    unsigned char* buf = smem + 16 * W + (size_t)(2 * w + half) * (16 * (size_t)cap + 16);
    float* Ds = reinterpret_cast<float*>(buf + 12 * (size_t)cap + 16);
    const uint32_t bar = dev::smem_u32(&bars[2 * w + half]);
    if (hl == 0) {
        dev::mbar_init(bar, 1);
        dev::fence_mbar_init();
    }
    __syncwarp();
    dev::pdl_wait();
    dev::pdl_launch_dependents();
    uint32_t phase = 0;   // of this half's barrier
    bool halted = false;  // a timeout was seen: leave the remaining items undone

    const int npairs = (a.n_items + 1) / 2;
    const int nwarps = gridDim.x * W;
    int pair = a.counter ? dev::queue_next_of(a.counter, npairs, nwarps, lane) : blockIdx.x * W + w;

    while (pair < npairs) {
        if (!halted) {
            const int item = 2 * pair + half;
            const bool has = item < a.n_items;  // the last pair's second half may be empty
            ItemDesc d{};
            d.n = 1;
            if (has) d = dev::load_item(a, item);
            const int n = dev::checked(d.n, 1, cap + 1, a.status);

            // ---- stage-in, one bulk copy per half
            dev::fence_proxy_async_smem();
            __syncwarp();
            bool bulk = false;
            const float* pts = reinterpret_cast<const float*>(buf);
            if (has)
                pts = dev::stage_points(a.xyz + 3 * d.src, n, buf, bar, hl == 0, hl, 16, &bulk,
                                        (a.stall & STALL_COPY) != 0, a.host_resident != 0);
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
            halted = __any_sync(dev::kFull, late || dev::is_timeout(seen));
            if (!halted) {
                // Both halves run every step below in lockstep (no branch that
                // differs between them inside the loops), each on its own
                // data; a half without work (no item, its rounds done, no
                // stride phase) computes on its own buffer and stores nothing.
                const int rows = (n + 15) >> 4;
                unsigned rmb[R], rmi[R];  // cached maxima of 16-point rows
#pragma unroll
                for (int s = 0; s < R; ++s) {
                    const int r = hl + 16 * s;
                    rmb[s] = r < rows ? __float_as_uint(1e10f) : 0u;
                    rmi[s] = r < rows ? (unsigned)(16 * r) : 0xffffffffu;
                }
                int32_t* out = a.out + d.dst;
                const int c = has ? dev::checked(d.c, 1, n + 1, a.status) : 0;
                const int kl = d.kl;
                const int kr = d.kr;
                int p = dev::checked(d.first, 0, n, a.status);
                int obuf = hl == 0 ? d.lo + p : 0;
                if (has && hl == 0 && !ROWS) out[0] = d.lo + p;
                int t = 1;
                // stride phase, as in the full-warp kernel, over 16-point rows
                const bool sp = has && p <= kl && kl <= kr;
                const int q = kr + 1;
                const dev::SmallDiv divq((uint32_t)q);
                const int x = n - 1 - kr - p;
                const int ts = x <= 0 ? 1 : (int)divq((uint32_t)(x + q - 1)) + 1;
                const int tn = min(ts, c);
                const int tw = min(ts, c - 1);
                bool ok = true;
                const int srows = sp ? rows : 0;
                const int rmax = max(srows, __shfl_xor_sync(dev::kFull, srows, 16));
                for (int i = 0; i < rmax; ++i) {
                    const bool ract = i < srows;
                    const int j = 16 * i + hl;
                    const int jc = min(j, n - 1);
                    const float px = pts[3 * jc], py = pts[3 * jc + 1], pz = pts[3 * jc + 2];
                    const int u = (int)divq((uint32_t)(max(jc + kl - p, 0)));
                    const int s1 = p + u * q, s0 = s1 - q;
                    const bool in1 = ract && j < n && u < tw && jc <= s1 + kr;
                    const bool in0 = ract && j < n && u >= 1 && u - 1 < tw && jc <= s0 + kr;
                    const int c1 = dev::checked(in1 ? s1 : jc, 0, n, a.status);
                    const int c0 = dev::checked(in0 ? s0 : jc, 0, n, a.status);
                    const float d1 = dev::sqdist(px, py, pz, pts[3 * c1], pts[3 * c1 + 1],
                                                 pts[3 * c1 + 2]);
                    const float d0 = dev::sqdist(px, py, pz, pts[3 * c0], pts[3 * c0 + 1],
                                                 pts[3 * c0 + 2]);
                    ok = ok && (!in1 || d1 < 1e10f) && (!in0 || d0 < 1e10f);
                    float v = j < n ? 1e10f : 0.f;
                    v = in1 ? fminf(v, d1) : v;
                    v = in0 ? fminf(v, d0) : v;
                    if (ract) Ds[j] = v;
                    const unsigned b = __float_as_uint(v);
                    const unsigned m = half_max(b, half);
                    const unsigned l = half_first(b == m, hmask, half);
                    if (ract) set_row<R>(rmb, rmi, i, m, (unsigned)(16 * i) + l, hl, 16);
                }
                const bool stride_ok = sp && (__ballot_sync(dev::kFull, !ok) & hmask) == 0u;
                if (stride_ok) {
                    if (ROWS) {
                        for (int r0 = 0; r0 + 16 <= tn; r0 += 16)
                            out[r0 + hl] = d.lo + p + (r0 + hl) * q;
                        obuf = d.lo + p + (((tn - 1) & ~15) + hl) * q;
                    } else {
                        for (int tt = 1 + hl; tt < tn; tt += 16) out[tt] = d.lo + p + tt * q;
                    }
                    p += (tn - 1) * q;
                    t = tn;
                } else {
                    if (sp) {  // the stride test failed: start again from 1e10
#pragma unroll
                        for (int s = 0; s < R; ++s) {
                            const int r = hl + 16 * s;
                            rmb[s] = r < rows ? __float_as_uint(1e10f) : 0u;
                            rmi[s] = r < rows ? (unsigned)(16 * r) : 0xffffffffu;
                        }
                    }
                    for (int j = hl; j < 16 * rows; j += 16) Ds[j] = j < n ? 1e10f : 0.f;
                }
                __syncwarp();
                const int nm1 = n - 1;
#pragma unroll 4
                while (__any_sync(dev::kFull, t < c)) {
                    const bool act = t < c;
                    const int wl = max(p - kl, 0);
                    const int wh = min(p + kr, nm1);
                    // the sample's neighbours, one per lane (past the end: the
                    // last point again, the same value); the sample itself: +0
                    int j = wl + hl;
                    j = min(j + (j >= p ? 1 : 0), wh);
                    const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
                    const float dd = dev::sqdist(pts[3 * j], pts[3 * j + 1], pts[3 * j + 2],
                                                 qx, qy, qz);
                    const float dn = fminf(Ds[j], dd);
                    if (act) Ds[j] = dn;
                    if (act && hl == 0) Ds[p] = 0.f;
                    __syncwarp();
                    const int r0 = wl >> 4, r1 = wh >> 4;
                    const unsigned b0 = __float_as_uint(Ds[16 * r0 + hl]);
                    const unsigned b1 = __float_as_uint(Ds[16 * r1 + hl]);
                    const unsigned m0 = half_max(b0, half);
                    const unsigned m1 = half_max(b1, half);
                    const unsigned l0 = half_first(b0 == m0, hmask, half);
                    const unsigned l1 = half_first(b1 == m1, hmask, half);
                    if (act) {
                        set_row<R>(rmb, rmi, r0, m0, (unsigned)(16 * r0) + l0, hl, 16);
                        set_row<R>(rmb, rmi, r1, m1, (unsigned)(16 * r1) + l1, hl, 16);
                    }
                    unsigned cb = rmb[0], ci = rmi[0];
#pragma unroll
                    for (int s = 1; s < R; ++s) {
                        const bool gt = rmb[s] > cb;
                        cb = gt ? rmb[s] : cb;
                        ci = gt ? rmi[s] : ci;
                    }
                    const unsigned mx = half_max(cb, half);
                    const int pn = (int)half_min(cb == mx ? ci : 0xffffffffu, half);
                    if (act) {
                        p = dev::checked(pn, 0, n, a.status);
                        if (ROWS) {
                            obuf = hl == (t & 15) ? d.lo + p : obuf;
                            if ((t & 15) == 15) out[(t & ~15) + hl] = obuf;
                        } else if (hl == 0) {
                            out[t] = d.lo + p;
                        }
                        ++t;
                    }
                }
                if (ROWS && has && hl <= ((c - 1) & 15)) out[((c - 1) & ~15) + hl] = obuf;
            }
        }
        __syncwarp();
        pair = a.counter ? dev::queue_next_of(a.counter, npairs, nwarps, lane) : pair + nwarps;
    }
}

using SectorKernel = void (*)(LaunchArgs);

// Kernel for sectors of up to 32 * rows points (rows <= kWinMaxRows).
// Pair kernel for sectors of up to 16 * rows16 points (16-point rows).
SectorKernel win2_kernel_for(int rows16, bool host_rows) {
    const int slots = (rows16 + 15) / 16;
    if (slots <= 1) return host_rows ? afps_win2_kernel<1, true> : afps_win2_kernel<1, false>;
    if (slots <= 2) return host_rows ? afps_win2_kernel<2, true> : afps_win2_kernel<2, false>;
    if (slots <= 4) return host_rows ? afps_win2_kernel<4, true> : afps_win2_kernel<4, false>;
    if (slots <= 8) return host_rows ? afps_win2_kernel<8, true> : afps_win2_kernel<8, false>;
    return nullptr;
}

SectorKernel win_kernel_for(int rows, bool host_rows, bool lean) {
#define AFPS_WIN_CASE(RR)                                                                      \
    if (host_rows)                                                                             \
        return lean ? afps_win_kernel<RR, true, true> : afps_win_kernel<RR, true, false>;      \
    return lean ? afps_win_kernel<RR, false, true> : afps_win_kernel<RR, false, false>;
    const int slots = (rows + 31) / 32;
    if (slots <= 1) { AFPS_WIN_CASE(1) }
    if (slots <= 2) { AFPS_WIN_CASE(2) }
    if (slots <= 4) { AFPS_WIN_CASE(4) }
    if (slots <= 8) { AFPS_WIN_CASE(8) }
#undef AFPS_WIN_CASE
    return nullptr;
}

}  // namespace afps
