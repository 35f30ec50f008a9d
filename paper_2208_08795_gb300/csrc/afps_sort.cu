// afps_sort.cu -- stable sort of each cloud's points by a key, on the device.
//
// AFPS and NPDU rely on dimensional locality (Sec. III-A): points stored
// next to each other should be close along some axis.  For input without it
// the paper suggests binning or sorting; this kernel sorts exactly.  One CTA
// per cloud runs a least-significant-digit radix sort of 32-bit keys in four
// 8-bit passes.  In each pass every warp owns a contiguous segment of the
// cloud and walks it 32 elements at a time: __match_any_sync groups the lanes
// holding the same digit, which gives each element its rank among equal
// digits and lets one lane per group advance the warp's counter for that
// digit (per-warp counters in shared memory).  A scan over (digit, warp)
// turns the counts into output offsets, and a second walk scatters the
// (key, index) pairs.  Ranks follow lane, chunk and warp order, so each pass
// is stable, and so is the sort: equal keys keep their storage order.
// Finally the points are gathered in sorted order with the permutation.
// Clouds of more than 4096 points (up to 16 x 12,288) are sorted by the
// cluster kernel further down instead, across 16 SMs.
//
// Keys: x, y or z; or the "diamond angle", a monotone stand-in for the
// azimuth atan2(y, x) on [0, 4) built from separately rounded additions and
// one division, which host code can reproduce exactly.  -0 is folded into +0
// before the float bits are made order-preserving as unsigned integers.
#include <mutex>
#include <set>

#include "afps_device.cuh"

namespace afps {

__device__ __forceinline__ float diamond_angle(float x, float y) {
    if (x == 0.f && y == 0.f) return 0.f;
    if (y >= 0.f) {
        if (x >= 0.f) return __fdiv_rn(y, __fadd_rn(x, y));
        return __fsub_rn(1.f, __fdiv_rn(x, __fadd_rn(-x, y)));
    }
    if (x < 0.f) return __fsub_rn(2.f, __fdiv_rn(y, __fsub_rn(-x, y)));
    return __fadd_rn(3.f, __fdiv_rn(x, __fsub_rn(x, y)));
}

__device__ __forceinline__ uint32_t sort_key_bits(const float* p, int key) {
    float k = key < 3 ? p[key] : diamond_angle(p[0], p[1]);
    k = __fadd_rn(k, 0.f);  // -0 -> +0
    const uint32_t u = __float_as_uint(k);
    return u ^ ((u >> 31) ? 0xffffffffu : 0x80000000u);  // ascending as unsigned
}

__global__ void __launch_bounds__(1024) afps_sort_kernel(
    const SortDesc* __restrict__ descs, const float* __restrict__ xyz, int key,
    uint32_t* __restrict__ keys_a, int32_t* __restrict__ idx_a, uint32_t* __restrict__ keys_b,
    int32_t* __restrict__ idx_b, float* __restrict__ xyz_out, int32_t* __restrict__ perm) {
    constexpr int kW = 32;                  // warps per CTA
    __shared__ uint32_t cnt[kW][257];       // per-warp digit counters (row padded)
    __shared__ uint32_t dbase[256];         // first output slot of each digit
    const SortDesc d = descs[blockIdx.x];
    const int n = d.n;
    const int64_t off = d.off;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int seg = ((n + 32 * kW - 1) / (32 * kW)) * 32;  // multiple of 32
    const int s0 = min(n, w * seg), s1 = min(n, s0 + seg);

    for (int i = tid; i < n; i += blockDim.x) {
        keys_a[off + i] = sort_key_bits(xyz + 3 * (off + i), key);
        idx_a[off + i] = i;
    }
    __syncthreads();

    uint32_t* sk = keys_a;
    int32_t* si = idx_a;
    uint32_t* dk = keys_b;
    int32_t* di = idx_b;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        for (int i = tid; i < kW * 257; i += blockDim.x) (&cnt[0][0])[i] = 0u;
        __syncthreads();
        // count this warp's digits
        for (int c = s0; c < s1; c += 32) {
            const int i = c + lane;
            const bool valid = i < s1;
            const uint32_t k = valid ? sk[off + i] : 0u;
            const uint32_t dg = valid ? (k >> shift) & 255u : 256u + lane;
            const unsigned m = __match_any_sync(dev::kFull, dg);
            if (valid && lane == __ffs(m) - 1) cnt[w][dg] += __popc(m);
            __syncwarp();
        }
        __syncthreads();
        // per digit: warps' exclusive prefix, then the digit totals' prefix
        if (tid < 256) {
            uint32_t s = 0;
            for (int q = 0; q < kW; ++q) {
                const uint32_t c = cnt[q][tid];
                cnt[q][tid] = s;
                s += c;
            }
            dbase[tid] = s;
        }
        __syncthreads();
        if (w == 0) {
            uint32_t v[8], run = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = dbase[8 * lane + u];
                run += v[u];
            }
            uint32_t incl = run;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(dev::kFull, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t base = incl - run;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                dbase[8 * lane + u] = base;
                base += v[u];
            }
        }
        __syncthreads();
        // scatter, stable within the warp's segment
        for (int c = s0; c < s1; c += 32) {
            const int i = c + lane;
            const bool valid = i < s1;
            const uint32_t k = valid ? sk[off + i] : 0u;
            const int32_t id = valid ? si[off + i] : 0;
            const uint32_t dg = valid ? (k >> shift) & 255u : 256u + lane;
            const unsigned m = __match_any_sync(dev::kFull, dg);
            const int leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (valid && lane == leader) {
                base = cnt[w][dg];
                cnt[w][dg] = base + __popc(m);
            }
            base = __shfl_sync(dev::kFull, base, leader);
            if (valid) {
                const uint32_t pos = dbase[dg] + base + __popc(m & lt_mask);
                dk[off + pos] = k;
                di[off + pos] = id;
            }
            __syncwarp();
        }
        __syncthreads();
        uint32_t* tk = sk;
        sk = dk;
        dk = tk;
        int32_t* ti = si;
        si = di;
        di = ti;
    }

    for (int i = tid; i < n; i += blockDim.x) {
        const int32_t j = si[off + i];
        perm[off + i] = j;
        const float* src = xyz + 3 * (off + j);
        float* dst = xyz_out + 3 * (off + i);
        dst[0] = src[0];
        dst[1] = src[1];
        dst[2] = src[2];
    }
}

// ---------------------------------------------------------------- clusters
// A large cloud is sorted by a thread-block cluster of kSortCS CTAs that
// keeps it in distributed shared memory: CTA r holds positions
// [r * chunk, (r + 1) * chunk) of the current order as (key, index) pairs.
// Each 8-bit pass counts digits per warp (as above), sends the CTA's 256
// digit totals to every CTA of the cluster, and after one cluster barrier
// every CTA knows, for each digit, the elements before it in lower digits
// and in lower CTAs; the scatter then stores each pair straight into the
// shared memory of the CTA that owns its new position, and a second
// cluster barrier ends the pass.  Ranks follow (digit, CTA, warp, chunk,
// lane) order, i.e. the current order, so every pass is stable.
constexpr int kSortCS = 16;  // CTAs per cluster (non-portable size)
constexpr int kSortCW = 16;  // warps per CTA
// Pairs per CTA at most: two buffers of them plus the counters fill the
// 227 KB of shared memory a CTA can have.
constexpr int kSortClusterChunk = 12288;

__global__ void __launch_bounds__(32 * kSortCW) afps_sort_cluster_kernel(
    const SortDesc* __restrict__ descs, const float* __restrict__ xyz, int key, int chunk,
    float* __restrict__ xyz_out, int32_t* __restrict__ perm) {
    extern __shared__ __align__(16) unsigned char smem[];
    constexpr int CS = kSortCS, W = kSortCW;
    uint2* pa = reinterpret_cast<uint2*>(smem);                     // chunk pairs
    uint2* pb = pa + chunk;                                          // chunk pairs
    uint32_t* cnt = reinterpret_cast<uint32_t*>(pb + chunk);         // [W][257]
    uint32_t* ctot = cnt + W * 257;                                  // [CS][256], from peers
    uint32_t* dbase = ctot + CS * 256;                               // [256]
    uint32_t* before = dbase + 256;                                  // [256]
    const int rank = (int)dev::cluster_ctarank();
    const SortDesc d = descs[dev::cluster_id_x()];
    const int n = d.n;
    const int64_t off = d.off;
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const unsigned lt_mask = (1u << lane) - 1u;
    const int c0 = rank * chunk;
    const int cn = max(0, min(n - c0, chunk));  // pairs this CTA holds
    const int seg = ((cn + 32 * W - 1) / (32 * W)) * 32;
    const int s0 = min(cn, w * seg), s1 = min(cn, s0 + seg);

    for (int i = tid; i < cn; i += blockDim.x)
        pa[i] = make_uint2(sort_key_bits(xyz + 3 * (off + c0 + i), key), (uint32_t)(c0 + i));
    __syncthreads();
    dev::cluster_sync();  // every CTA of the cluster is running before remote stores

    uint2* src = pa;
    uint2* dst = pb;
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        for (int i = tid; i < W * 257; i += blockDim.x) cnt[i] = 0u;
        __syncthreads();
        for (int c = s0; c < s1; c += 32) {
            const int i = c + lane;
            const bool valid = i < s1;
            const uint32_t k = valid ? src[i].x : 0u;
            const uint32_t dg = valid ? (k >> shift) & 255u : 256u + lane;
            const unsigned m = __match_any_sync(dev::kFull, dg);
            if (valid && lane == __ffs(m) - 1) cnt[w * 257 + dg] += __popc(m);
            __syncwarp();
        }
        __syncthreads();
        // per digit: the warps' exclusive prefix, and the CTA's total to every CTA
        if (tid < 256) {
            uint32_t t = 0;
            for (int q = 0; q < W; ++q) {
                const uint32_t c = cnt[q * 257 + tid];
                cnt[q * 257 + tid] = t;
                t += c;
            }
            const uint32_t slot = dev::smem_u32(&ctot[rank * 256 + tid]);
            for (int r = 0; r < CS; ++r)
                asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(dev::mapa(slot, (uint32_t)r)),
                             "r"(t)
                             : "memory");
        }
        dev::cluster_sync();
        // per digit: elements of lower CTAs, and all of them
        if (tid < 256) {
            uint32_t b = 0, all = 0;
            for (int r = 0; r < CS; ++r) {
                const uint32_t v = ctot[r * 256 + tid];
                b += r < rank ? v : 0u;
                all += v;
            }
            before[tid] = b;
            dbase[tid] = all;
        }
        __syncthreads();
        if (w == 0) {  // exclusive scan of the digit totals
            uint32_t v[8], run = 0;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                v[u] = dbase[8 * lane + u];
                run += v[u];
            }
            uint32_t incl = run;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(dev::kFull, incl, o);
                if (lane >= o) incl += t;
            }
            uint32_t base = incl - run;
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                dbase[8 * lane + u] = base + before[8 * lane + u];
                base += v[u];
            }
        }
        __syncthreads();
        // scatter into the owner CTA's buffer
        for (int c = s0; c < s1; c += 32) {
            const int i = c + lane;
            const bool valid = i < s1;
            const uint2 kv = valid ? src[i] : make_uint2(0u, 0u);
            const uint32_t dg = valid ? (kv.x >> shift) & 255u : 256u + lane;
            const unsigned m = __match_any_sync(dev::kFull, dg);
            const int leader = __ffs(m) - 1;
            uint32_t base = 0;
            if (valid && lane == leader) {
                base = cnt[w * 257 + dg];
                cnt[w * 257 + dg] = base + __popc(m);
            }
            base = __shfl_sync(dev::kFull, base, leader);
            if (valid) {
                const uint32_t pos = dbase[dg] + base + __popc(m & lt_mask);  // < n
                const uint32_t owner = pos / (uint32_t)chunk;
                const uint32_t at = dev::smem_u32(&dst[pos - owner * (uint32_t)chunk]);
                asm volatile("st.shared::cluster.v2.u32 [%0], {%1, %2};" ::"r"(dev::mapa(at, owner)),
                             "r"(kv.x), "r"(kv.y)
                             : "memory");
            }
            __syncwarp();
        }
        dev::cluster_sync();  // every pair of the pass has landed
        uint2* t = src;
        src = dst;
        dst = t;
    }

    for (int i = tid; i < cn; i += blockDim.x) {
        const int32_t j = (int32_t)src[i].y;
        perm[off + c0 + i] = j;
        const float* a = xyz + 3 * (off + j);
        float* b = xyz_out + 3 * (off + c0 + i);
        b[0] = a[0];
        b[1] = a[1];
        b[2] = a[2];
    }
}

int sort_cluster_capacity() { return kSortCS * kSortClusterChunk; }

cudaError_t launch_sort(const SortDesc* d_descs, int32_t B, const float* xyz, int key,
                        uint32_t* keys_a, int32_t* idx_a, uint32_t* keys_b, int32_t* idx_b,
                        float* xyz_out, int32_t* perm, cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    afps_sort_kernel<<<B, 1024, 0, stream>>>(d_descs, xyz, key, keys_a, idx_a, keys_b, idx_b,
                                             xyz_out, perm);
    return cudaGetLastError();
}

cudaError_t launch_sort_cluster(const SortDesc* d_descs, int32_t B, int32_t max_n,
                                const float* xyz, int key, float* xyz_out, int32_t* perm,
                                cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    const int chunk = ((max_n + kSortCS - 1) / kSortCS + 31) / 32 * 32;
    if (chunk > kSortClusterChunk) return cudaErrorInvalidValue;
    const size_t smem = 2 * (size_t)chunk * sizeof(uint2) +
                        sizeof(uint32_t) * ((size_t)kSortCW * 257 + kSortCS * 256 + 512);
    {  // function attributes, once per device
        static std::mutex mu;
        static std::set<int> done;
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        std::lock_guard<std::mutex> lock(mu);
        if (!done.count(dev)) {
            e = cudaFuncSetAttribute(afps_sort_cluster_kernel,
                                     cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
            if (e == cudaSuccess)
                e = cudaFuncSetAttribute(afps_sort_cluster_kernel,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(2 * (size_t)kSortClusterChunk * sizeof(uint2) +
                                               sizeof(uint32_t) *
                                                   ((size_t)kSortCW * 257 + kSortCS * 256 + 512)));
            if (e != cudaSuccess) return e;
            done.insert(dev);
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(B * kSortCS), 1, 1);
    cfg.blockDim = dim3(32 * kSortCW, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = kSortCS;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, afps_sort_cluster_kernel, d_descs, xyz, key, chunk, xyz_out,
                              perm);
}

}  // namespace afps
