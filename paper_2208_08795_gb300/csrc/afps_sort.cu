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
//
// Keys: x, y or z; or the "diamond angle", a monotone stand-in for the
// azimuth atan2(y, x) on [0, 4) built from separately rounded additions and
// one division, which host code can reproduce exactly.  -0 is folded into +0
// before the float bits are made order-preserving as unsigned integers.
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

cudaError_t launch_sort(const SortDesc* d_descs, int32_t B, const float* xyz, int key,
                        uint32_t* keys_a, int32_t* idx_a, uint32_t* keys_b, int32_t* idx_b,
                        float* xyz_out, int32_t* perm, cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    afps_sort_kernel<<<B, 1024, 0, stream>>>(d_descs, xyz, key, keys_a, idx_a, keys_b, idx_b,
                                             xyz_out, perm);
    return cudaGetLastError();
}

}  // namespace afps
