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
//   emit       sample indices are buffered one per lane and stored as one
//              coalesced 128-byte row every 32 iterations.
// Work items come from a device counter (dynamic queue) or by static
// striding.  No CTA-wide synchronisation: warps of a CTA are independent.
#include "afps_device.cuh"

namespace afps {

template <int P, bool NPDU>
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
    uint32_t phase = 0;

    const int nwarps = gridDim.x * W;
    int item;
    if (a.counter) {
        unsigned v = 0;
        if (lane == 0) v = atomicAdd(a.counter, 1u);
        item = (int)__shfl_sync(dev::kFull, v, 0);
    } else {
        item = blockIdx.x * W + w;
    }

    while (item < a.n_items) {
        const ItemDesc d = dev::load_item(a, item);
        const int n = d.n;

        // ---- stage-in (the previous item's readers are done: fence + sync)
        dev::fence_proxy_async_smem();
        __syncwarp();
        bool bulk;
        const float* pts =
            dev::stage_points(a.xyz + 3 * d.src, n, buf, bar, lane == 0, lane, 32, &bulk,
                              a.stall_copy != 0);
        if (bulk) {
            if (!dev::mbar_wait_bounded(bar, phase, a.timeout_ns)) {
                dev::record_status(a.status, DEV_TIMEOUT_STAGE);
                if (!dev::mbar_wait_bounded(bar, phase, a.timeout_ns))
                    dev::record_status(a.status, DEV_TIMEOUT_DRAIN);
            }
            phase ^= 1u;
        }
        __syncwarp();

        float x[P], y[P], z[P], D[P];
#pragma unroll
        for (int i = 0; i < P; ++i) {
            const int j = lane + 32 * i;
            if (j < n) {
                x[i] = pts[3 * j];
                y[i] = pts[3 * j + 1];
                z[i] = pts[3 * j + 2];
                D[i] = 1e10f;
            } else {  // padding: distance +0 stays +0 and loses every tie
                x[i] = 0.f;
                y[i] = 0.f;
                z[i] = 0.f;
                D[i] = 0.f;
            }
        }

        int32_t* out = a.out + d.dst;
        const int c = d.c;
        const int kl = d.k >> 1;
        const int kr = d.k - kl;
        int p = d.first;
        int obuf = 0;
        for (int t = 0; t < c; ++t) {
            if (lane == (t & 31)) obuf = d.lo + p;
            if ((t & 31) == 31 || t == c - 1) {
                if (lane <= (t & 31)) out[(t & ~31) + lane] = obuf;
            }
            if (t == c - 1) break;

            const float qx = pts[3 * p], qy = pts[3 * p + 1], qz = pts[3 * p + 2];
            const int wlo = p - kl, whi = p + kr;
            float best = -1.f;
            int bi = 0;
#pragma unroll
            for (int i = 0; i < P; ++i) {
                if (32 * i < n) {  // warp-uniform: the row holds real points
                    if (NPDU) {
                        if (32 * i + 31 >= wlo && 32 * i <= whi) {  // row meets the window
                            const int j = lane + 32 * i;
                            if (j >= wlo && j <= whi && j < n)
                                D[i] = fminf(D[i], dev::sqdist(x[i], y[i], z[i], qx, qy, qz));
                        }
                    } else {
                        D[i] = fminf(D[i], dev::sqdist(x[i], y[i], z[i], qx, qy, qz));
                    }
                    if (D[i] > best) {  // strict: lowest row wins ties
                        best = D[i];
                        bi = i;
                    }
                }
            }
            const unsigned bits = __float_as_uint(best);
            const unsigned m = __reduce_max_sync(dev::kFull, bits);
            const unsigned cand = bits == m ? (unsigned)(lane + 32 * bi) : 0xffffffffu;
            p = (int)__reduce_min_sync(dev::kFull, cand);
        }

        if (a.counter) {
            unsigned v = 0;
            if (lane == 0) v = atomicAdd(a.counter, 1u);
            item = (int)__shfl_sync(dev::kFull, v, 0);
        } else {
            item += nwarps;
        }
    }
}

using SectorKernel = void (*)(LaunchArgs);

SectorKernel warp_kernel_for(int P, bool npdu) {
#define AFPS_WARP_CASE(PP) \
    case PP:               \
        return npdu ? afps_warp_kernel<PP, true> : afps_warp_kernel<PP, false>;
    switch (P) {
        AFPS_WARP_CASE(1)
        AFPS_WARP_CASE(2)
        AFPS_WARP_CASE(3)
        AFPS_WARP_CASE(4)
        AFPS_WARP_CASE(6)
        AFPS_WARP_CASE(8)
        AFPS_WARP_CASE(12)
        AFPS_WARP_CASE(16)
        default:
            return nullptr;
    }
#undef AFPS_WARP_CASE
}

}  // namespace afps
