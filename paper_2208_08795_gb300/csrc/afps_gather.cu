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

// Frame copies of a serving step: grid.y = frame, grid.x = 16 KB chunks of
// it; 16-byte vectors where both ends allow, else 4-byte words.  The
// descriptors travel in the kernel's parameters, so a step's admission is
// one launch instead of a copy call per frame.
__global__ void __launch_bounds__(256) afps_frame_copy_kernel(const __grid_constant__ FrameCopyBatch b) {
    const int f = blockIdx.y;
    if (f >= b.n) return;
    const FrameCopy c = b.c[f];
    constexpr int64_t kChunk = 16384;
    const int64_t lo = (int64_t)blockIdx.x * kChunk;
    if (lo >= c.bytes) return;
    const int64_t hi = min(c.bytes, lo + kChunk);
    const char* src = static_cast<const char*>(c.src);
    char* dst = static_cast<char*>(c.dst);
    const bool vec = ((reinterpret_cast<uintptr_t>(src) | reinterpret_cast<uintptr_t>(dst)) & 15) == 0;
    if (vec) {
        const int64_t v_hi = lo + ((hi - lo) & ~int64_t(15));
        for (int64_t o = lo + 16 * threadIdx.x; o < v_hi; o += 16 * blockDim.x)
            *reinterpret_cast<uint4*>(dst + o) = *reinterpret_cast<const uint4*>(src + o);
        for (int64_t o = v_hi + 4 * threadIdx.x; o < hi; o += 4 * blockDim.x)
            *reinterpret_cast<uint32_t*>(dst + o) = *reinterpret_cast<const uint32_t*>(src + o);
    } else {
        for (int64_t o = lo + 4 * threadIdx.x; o < hi; o += 4 * blockDim.x)
            *reinterpret_cast<uint32_t*>(dst + o) = *reinterpret_cast<const uint32_t*>(src + o);
    }
}

cudaError_t launch_frame_copy(const FrameCopyBatch& batch, int64_t max_bytes, cudaStream_t stream) {
    if (batch.n < 1) return cudaSuccess;
    const dim3 grid((unsigned)((max_bytes + 16383) / 16384), (unsigned)batch.n, 1);
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
