// afps_gather.cu -- gather between chained sampling levels.
//
// The PointNet++ hierarchy the paper accelerates (Sec. I-II) samples each
// level from the previous level's samples.  The next level's cloud is the
// previous samples taken in ascending storage index, which preserves the
// storage order and so the dimensional locality that AFPS and NPDU rely on
// (Sec. III-A).  One CTA per cloud: a counting sort over the cloud's n points
// (16-bit counters in shared memory, two per word) and a block-wide exclusive
// scan give every sample its destination; each thread writes the source index
// of the samples in its range of points to their destinations, then all
// threads copy points and original frame indices for consecutive
// destinations in parallel.  Counting (not flags) keeps repeated indices,
// should a degenerate cloud produce any.  The output xyz must not overlap the
// input.
#include <algorithm>
#include <mutex>
#include <set>

#include "afps_device.cuh"

namespace afps {

__global__ void __launch_bounds__(1024) afps_gather_kernel(
    const GatherDesc* __restrict__ descs, const float* __restrict__ in_xyz,
    const int32_t* __restrict__ in_frame, const int32_t* __restrict__ sel,
    float* __restrict__ out_xyz, int32_t* __restrict__ out_frame,
    int32_t* __restrict__ sel_frame) {
    extern __shared__ __align__(16) uint32_t cnt[];  // (n + 1) / 2 words of two 16-bit counters
    __shared__ uint32_t warp_sum[32];
    __shared__ uint32_t total;
    const GatherDesc d = descs[blockIdx.x];
    const int T = blockDim.x, tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = d.n, c = d.c;
    const int words = (n + 1) >> 1;

    // 1. count the samples of every point
    for (int i = tid; i < words; i += T) cnt[i] = 0u;
    __syncthreads();
    constexpr int kBatch = 8;  // loads in flight per thread
    for (int s0 = 0; s0 < c; s0 += kBatch * T) {
        int jv[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int s = s0 + u * T + tid;
            jv[u] = s < c ? sel[d.sel + s] : -1;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u)
            if (jv[u] >= 0 && jv[u] < n) atomicAdd(&cnt[jv[u] >> 1], 1u << (16 * (jv[u] & 1)));
    }
    __syncthreads();

    // 2. exclusive scan over points; thread t owns points [j0, j1)
    const int per = (n + T - 1) / T;
    const int j0 = min(n, tid * per), j1 = min(n, j0 + per);
    uint32_t local = 0;
    for (int j = j0; j < j1; ++j) local += (cnt[j >> 1] >> (16 * (j & 1))) & 0xffffu;
    uint32_t incl = local;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t v = __shfl_up_sync(dev::kFull, incl, o);
        if (lane >= o) incl += v;
    }
    if (lane == 31) warp_sum[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = T >> 5;
        const uint32_t v = lane < nw ? warp_sum[lane] : 0u;
        uint32_t inc = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(dev::kFull, inc, o);
            if (lane >= o) inc += u;
        }
        if (lane < nw) warp_sum[lane] = inc - v;  // exclusive prefix of warps
        if (lane == nw - 1) total = inc;
    }
    __syncthreads();

    // 3. destination of every sample: its point index goes into the first
    //    word of the destination's xyz slot (overwritten in step 4)
    int32_t* slot = reinterpret_cast<int32_t*>(out_xyz) + 3 * d.out_xyz;
    uint32_t pos = warp_sum[w] + incl - local;
    for (int j = j0; j < j1; ++j) {
        for (uint32_t k = (cnt[j >> 1] >> (16 * (j & 1))) & 0xffffu; k; --k, ++pos)
            slot[3 * pos] = j;
    }
    __syncthreads();

    // 4. all threads copy consecutive destinations, kBatch loads in flight
    const int m = (int)total;
    for (int i0 = 0; i0 < m; i0 += kBatch * T) {
        int jv[kBatch];
        float px[kBatch], py[kBatch], pz[kBatch];
        int32_t fr[kBatch];
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = i0 + u * T + tid;
            jv[u] = i < m ? slot[3 * i] : 0;
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const float* src = in_xyz + 3 * (d.in_xyz + jv[u]);
            px[u] = src[0];
            py[u] = src[1];
            pz[u] = src[2];
            fr[u] = d.in_frame >= 0 ? in_frame[d.in_frame + jv[u]] : jv[u];
        }
#pragma unroll
        for (int u = 0; u < kBatch; ++u) {
            const int i = i0 + u * T + tid;
            if (i < m) {
                float* dst = out_xyz + 3 * (d.out_xyz + i);
                dst[0] = px[u];
                dst[1] = py[u];
                dst[2] = pz[u];
                if (d.out_frame >= 0) out_frame[d.out_frame + i] = fr[u];
            }
        }
    }

    // 5. frame index of every sample in its own (emission) order
    if (d.sel_frame >= 0) {
        for (int s0 = 0; s0 < c; s0 += kBatch * T) {
            int jv[kBatch];
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int s = s0 + u * T + tid;
                jv[u] = s < c ? sel[d.sel + s] : -1;
            }
#pragma unroll
            for (int u = 0; u < kBatch; ++u) {
                const int s = s0 + u * T + tid;
                if (s < c && jv[u] >= 0 && jv[u] < n)
                    sel_frame[d.sel_frame + s] = d.in_frame >= 0 ? in_frame[d.in_frame + jv[u]] : jv[u];
            }
        }
    }
}

// Frame copies of a serving step: grid.y = frame, grid.x = the CTAs sharing
// it, each thread with eight 16-byte loads in flight (4-byte words where an
// end is not 16-byte aligned).  The frames come from page-locked host memory
// over the C2C link, whose rate a few hundred KB in flight already reaches;
// so the copy keeps to about 128 CTAs of 256 threads in all, and leaves the
// SMs to the sampling launches of another stream meanwhile.  The descriptors
// travel in the kernel's parameters: a step's admission is one launch.
__global__ void __launch_bounds__(256) afps_frame_copy_kernel(const __grid_constant__ FrameCopyBatch b) {
    const int f = blockIdx.y;
    if (f >= b.n) return;
    const FrameCopy c = b.c[f];
    const char* src = static_cast<const char*>(c.src);
    char* dst = static_cast<char*>(c.dst);
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    int64_t tail = 0;  // first byte of the 4-byte-word part
    if (vec) {
        const uint4* s4 = reinterpret_cast<const uint4*>(src);
        uint4* d4 = reinterpret_cast<uint4*>(dst);
        const int64_t n16 = c.bytes / 16;
        int64_t i = t;
        for (; i + 7 * stride < n16; i += 8 * stride) {
            uint4 v[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) v[u] = s4[i + u * stride];
#pragma unroll
            for (int u = 0; u < 8; ++u) d4[i + u * stride] = v[u];
        }
        for (; i < n16; i += stride) d4[i] = s4[i];
        tail = 16 * n16;
    }
    for (int64_t o = tail + 4 * t; o < c.bytes; o += 4 * stride)
        *reinterpret_cast<uint32_t*>(dst + o) = *reinterpret_cast<const uint32_t*>(src + o);
}

cudaError_t launch_frame_copy(const FrameCopyBatch& batch, int64_t max_bytes, cudaStream_t stream) {
    if (batch.n < 1) return cudaSuccess;
    // about 128 CTAs in all, at most one per 32 KB of the largest frame
    const int64_t per_frame =
        std::max<int64_t>(1, std::min<int64_t>((max_bytes + 32767) / 32768, 128 / batch.n));
    const dim3 grid((unsigned)per_frame, (unsigned)batch.n, 1);
    afps_frame_copy_kernel<<<grid, 256, 0, stream>>>(batch);
    return cudaGetLastError();
}

cudaError_t launch_gather(const GatherDesc* d_descs, int32_t B, int32_t max_n,
                          const float* in_xyz, const int32_t* in_frame, const int32_t* sel,
                          float* out_xyz, int32_t* out_frame, int32_t* sel_frame,
                          cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    const size_t smem = 4 * (size_t)((max_n + 1) / 2) + 16;
    {  // the largest dynamic shared memory any cloud can need, once per device
        static std::mutex mu;
        static std::set<int> done;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (!done.count(dev)) {
            e = cudaFuncSetAttribute(reinterpret_cast<const void*>(afps_gather_kernel),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(4 * (size_t)((kGatherMaxPoints + 1) / 2) + 16));
            if (e != cudaSuccess) return e;
            done.insert(dev);
        }
    }
    afps_gather_kernel<<<B, 1024, smem, stream>>>(d_descs, in_xyz, in_frame, sel, out_xyz,
                                                  out_frame, sel_frame);
    return cudaGetLastError();
}

}  // namespace afps
