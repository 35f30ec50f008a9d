// afps_gather.cu -- gather between chained sampling levels.
//
// The PointNet++ hierarchy the paper accelerates (Sec. I-II) samples each
// level from the previous level's samples.  The next level's cloud is the
// previous samples taken in ascending storage index, which preserves the
// storage order and so the dimensional locality that AFPS and NPDU rely on
// (Sec. III-A).  One CTA per cloud: a counting sort over the cloud's n points
// (16-bit counters in shared memory, two per word), a block-wide exclusive
// scan, then a scatter of points and original frame indices in ascending
// order.  Counting (not flags) keeps repeated indices, should a degenerate
// cloud produce any.
#include "afps_device.cuh"

namespace afps {

__global__ void __launch_bounds__(1024) afps_gather_kernel(
    const GatherDesc* __restrict__ descs, const float* __restrict__ in_xyz,
    const int32_t* __restrict__ in_frame, const int32_t* __restrict__ sel,
    float* __restrict__ out_xyz, int32_t* __restrict__ out_frame,
    int32_t* __restrict__ sel_frame) {
    extern __shared__ __align__(16) uint32_t cnt[];  // (n + 1) / 2 words + 32 warp sums
    __shared__ uint32_t warp_sum[32];
    const GatherDesc d = descs[blockIdx.x];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = d.n, c = d.c;
    const int words = (n + 1) >> 1;

    for (int i = tid; i < words; i += T) cnt[i] = 0u;
    __syncthreads();
    for (int s = tid; s < c; s += T) {
        const int j = sel[d.sel + s];
        if (j >= 0 && j < n) {
            atomicAdd(&cnt[j >> 1], 1u << (16 * (j & 1)));
            if (d.sel_frame >= 0) sel_frame[d.sel_frame + s] = d.in_frame >= 0 ? in_frame[d.in_frame + j] : j;
        }
    }
    __syncthreads();

    // each thread owns points [j0, j1)
    const int per = (n + T - 1) / T;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    uint32_t local = 0;
    for (int j = j0; j < j1; ++j) local += (cnt[j >> 1] >> (16 * (j & 1))) & 0xffffu;
    // block exclusive scan of `local`
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(dev::kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = T >> 5;
        uint32_t v = lane < nw ? warp_sum[lane] : 0u;
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(dev::kFull, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane < nw) warp_sum[lane] = inc - v;  // exclusive prefix of warps
    }
    __syncthreads();
    uint32_t pos = warp_sum[w] + incl - local;

    for (int j = j0; j < j1; ++j) {
        uint32_t k = (cnt[j >> 1] >> (16 * (j & 1))) & 0xffffu;
        if (!k) continue;
        const float* src = in_xyz + 3 * (d.in_xyz + j);
        const float px = src[0], py = src[1], pz = src[2];
        const int32_t fr = d.in_frame >= 0 ? in_frame[d.in_frame + j] : j;
        for (; k; --k, ++pos) {
            float* dst = out_xyz + 3 * (d.out_xyz + pos);
            dst[0] = px;
            dst[1] = py;
            dst[2] = pz;
            if (d.out_frame >= 0) out_frame[d.out_frame + pos] = fr;
        }
    }
}

cudaError_t launch_gather(const GatherDesc* d_descs, int32_t B, int32_t max_n,
                          const float* in_xyz, const int32_t* in_frame, const int32_t* sel,
                          float* out_xyz, int32_t* out_frame, int32_t* sel_frame,
                          cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    const size_t smem = 4 * (size_t)((max_n + 1) / 2) + 16;
    cudaError_t e = cudaFuncSetAttribute(reinterpret_cast<const void*>(afps_gather_kernel),
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    afps_gather_kernel<<<B, 1024, smem, stream>>>(d_descs, in_xyz, in_frame, sel, out_xyz,
                                                  out_frame, sel_frame);
    return cudaGetLastError();
}

}  // namespace afps
