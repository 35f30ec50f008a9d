// afps_knn.cu -- k nearest neighbours: the other grouping step that follows
// sampling in point-cloud networks (Sec. I-II).
//
// For each centroid: the K points with the smallest key (squared distance
// bits, index), where the distance is the fp32 (dx*dx + dy*dy) + dz*dz with
// dx = point - centroid and every operation rounded on its own; ties go to
// the lower index; nearest first.
//
// One warp per centroid keeps the smallest keys seen so far sorted across
// its lanes: element l of the list lives in lane l % 32 of slot l / 32
// (S slots, K <= 32 S).  Each 32-point chunk ballots the points whose key is
// below the current K-th key, and they enter one at a time: the rank is the
// number of list keys below the new key (one ballot per slot) and the
// elements from the rank on move up by one (shuffles).  With one slot and
// many candidates the chunk is bitonic-sorted and merged instead.  Keys are
// unique (the index is part of them), so the first K elements equal the
// first K of the fully sorted keys whatever the scan order.
//
// On a cloud sorted ascending along `axis` (dimensional locality, Sec.
// III-A) the scan starts at the centroid's chunk and grows outward, nearer
// side first.  Past a boundary the rounded axis difference only grows in
// magnitude, and the rounded distance is at least the rounded square of that
// difference (every term is >= 0 and rounding is monotone), so a side stops
// once that square exceeds the K-th distance; the result equals the full
// scan's exactly.
#include "afps_device.cuh"

namespace afps {

constexpr int kKnnWarps = 8;
constexpr unsigned long long kNoKey = ~0ull;  // above every real key

__device__ __forceinline__ unsigned long long shfl64(unsigned long long v, int src) {
    const unsigned lo = __shfl_sync(dev::kFull, (unsigned)v, src);
    const unsigned hi = __shfl_sync(dev::kFull, (unsigned)(v >> 32), src);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long shfl64_up(unsigned long long v) {
    const unsigned lo = __shfl_up_sync(dev::kFull, (unsigned)v, 1);
    const unsigned hi = __shfl_up_sync(dev::kFull, (unsigned)(v >> 32), 1);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long shfl64_xor(unsigned long long v, int m) {
    const unsigned lo = __shfl_xor_sync(dev::kFull, (unsigned)v, m);
    const unsigned hi = __shfl_xor_sync(dev::kFull, (unsigned)(v >> 32), m);
    return ((unsigned long long)hi << 32) | lo;
}

__device__ __forceinline__ unsigned long long min64(unsigned long long a, unsigned long long b) {
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long max64(unsigned long long a, unsigned long long b) {
    return a < b ? b : a;
}

// Bitonic sort of one key per lane, ascending with the lane.
__device__ __forceinline__ unsigned long long warp_sort(unsigned long long v, int lane) {
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const unsigned long long o = shfl64_xor(v, j);
            // lower lane of an ascending block (or upper of a descending) keeps the min
            const bool keep_min = ((lane & j) == 0) == ((lane & k) == 0);
            v = keep_min ? min64(v, o) : max64(v, o);
        }
    }
    return v;
}

template <int S>
struct KnnList {
    unsigned long long key[S];
    unsigned long long thr;  // the K-th key (kNoKey while fewer than K are held)
    int kl, kslot;           // lane and slot of element K-1

    __device__ __forceinline__ void init(int K) {
#pragma unroll
        for (int s = 0; s < S; ++s) key[s] = kNoKey;
        thr = kNoKey;
        kslot = (K - 1) >> 5;
        kl = (K - 1) & 31;
    }

    // Insert key c (warp-uniform, c < thr).
    __device__ __forceinline__ void insert(unsigned long long c, int lane) {
        int pos = 0;
#pragma unroll
        for (int s = 0; s < S; ++s) pos += __popc(__ballot_sync(dev::kFull, key[s] < c));
        unsigned long long tail = 0;  // element 32 s - 1: lane 31 of the slot below
#pragma unroll
        for (int s = 0; s < S; ++s) {
            unsigned long long up = shfl64_up(key[s]);
            const unsigned long long next_tail = shfl64(key[s], 31);
            if (lane == 0) up = tail;
            const int l = 32 * s + lane;
            key[s] = l > pos ? up : (l == pos ? c : key[s]);
            tail = next_tail;
        }
        unsigned long long t = key[0];
#pragma unroll
        for (int s = 1; s < S; ++s) t = kslot == s ? key[s] : t;
        thr = shfl64(t, kl);
    }

    // One slot only: merge a whole chunk's keys (any order, one per lane).
    // The 32 smallest of list and chunk are the elementwise minimum of the
    // ascending list and the descending chunk (a bitonic sequence), which a
    // bitonic merge then sorts.
    __device__ __forceinline__ void merge(unsigned long long ck, int lane) {
        const unsigned long long c = shfl64(warp_sort(ck, lane), 31 - lane);
        unsigned long long v = min64(key[0], c);
#pragma unroll
        for (int j = 16; j > 0; j >>= 1) {
            const unsigned long long o = shfl64_xor(v, j);
            v = (lane & j) == 0 ? min64(v, o) : max64(v, o);
        }
        key[0] = v;
        thr = shfl64(v, kl);
    }
};

// Candidates in one chunk at or above which the one-slot list merges the
// whole chunk instead of inserting them one by one (a sort and a merge cost
// about as much as five insertions).
constexpr int kMergeAt = 6;

// Points [a, b) of the cloud (b - a <= 32) against the list.
template <int S>
__device__ __forceinline__ void knn_chunk(KnnList<S>& L, const float* P, int a, int b, float cx,
                                          float cy, float cz, int lane) {
    const int j = a + lane;
    unsigned long long ck = kNoKey;
    if (j < b) {
        const float d = dev::sqdist(P[3 * j], P[3 * j + 1], P[3 * j + 2], cx, cy, cz);
        ck = ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)j;
    }
    unsigned m = __ballot_sync(dev::kFull, ck < L.thr);
    if (S == 1 && __popc(m) >= kMergeAt) {
        L.merge(ck, lane);
        return;
    }
    while (m) {
        const int src = __ffs(m) - 1;
        m &= m - 1;
        const unsigned long long c = shfl64(ck, src);
        if (c < L.thr) L.insert(c, lane);
    }
}

template <int S>
__global__ void __launch_bounds__(32 * kKnnWarps) afps_knn_kernel(
    const GroupDesc* __restrict__ descs, const float* __restrict__ xyz,
    const int32_t* __restrict__ sel, int K, int axis, int32_t* __restrict__ out,
    float* __restrict__ dist2) {
    const GroupDesc d = descs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * kKnnWarps + (threadIdx.x >> 5);
    if (s >= d.c) return;  // warp-uniform
    const float* P = xyz + 3 * d.pt_off;
    const int n = d.n;
    const int ci = min(max(sel[d.sel_off + s], 0), n - 1);
    const float cx = P[3 * ci], cy = P[3 * ci + 1], cz = P[3 * ci + 2];
    KnnList<S> L;
    L.init(K);
    if (axis < 0) {
        for (int a = 0; a < n; a += 32) knn_chunk<S>(L, P, a, min(a + 32, n), cx, cy, cz, lane);
    } else {
        const float ca = axis == 0 ? cx : axis == 1 ? cy : cz;
        int lo = ci & ~31, hi = min(lo + 32, n);
        knn_chunk<S>(L, P, lo, hi, cx, cy, cz, lane);
        bool left = lo > 0, right = hi < n;  // sides still to scan (warp-uniform)
        while (left || right) {
            // squared axis distance of the nearest unscanned point on each side
            float gl = __int_as_float(0x7f800000), gr = gl;
            if (left) {
                const float e = __fsub_rn(P[3 * (lo - 1) + axis], ca);
                gl = __fmul_rn(e, e);
            }
            if (right) {
                const float e = __fsub_rn(P[3 * hi + axis], ca);
                gr = __fmul_rn(e, e);
            }
            if (L.thr != kNoKey) {  // K keys held: a side past the K-th distance is done
                const float kd = __uint_as_float((unsigned)(L.thr >> 32));
                left = left && !(gl > kd);
                right = right && !(gr > kd);
                if (!left && !right) break;
            }
            if (left && (!right || gl <= gr)) {
                const int a = max(lo - 32, 0);
                knn_chunk<S>(L, P, a, lo, cx, cy, cz, lane);
                lo = a;
                left = lo > 0;
            } else {
                const int b = min(hi + 32, n);
                knn_chunk<S>(L, P, hi, b, cx, cy, cz, lane);
                hi = b;
                right = hi < n;
            }
        }
    }
    int32_t* row = out + (d.sel_off + s) * (int64_t)K;
    float* drow = dist2 ? dist2 + (d.sel_off + s) * (int64_t)K : nullptr;
#pragma unroll
    for (int q = 0; q < S; ++q) {
        const int l = 32 * q + lane;
        if (l < K) {
            row[l] = (int32_t)(unsigned)L.key[q];
            if (drow) drow[l] = __uint_as_float((unsigned)(L.key[q] >> 32));
        }
    }
}

cudaError_t launch_knn(const GroupDesc* d_descs, int32_t B, int32_t max_c, const float* xyz,
                       const int32_t* sel, int32_t K, int32_t axis, int32_t* out, float* dist2,
                       cudaStream_t stream) {
    if (B < 1 || max_c < 1) return cudaSuccess;
    if (K < 1 || K > 64) return cudaErrorInvalidValue;
    const dim3 grid((unsigned)((max_c + kKnnWarps - 1) / kKnnWarps), (unsigned)B);
    if (K <= 32)
        afps_knn_kernel<1><<<grid, 32 * kKnnWarps, 0, stream>>>(d_descs, xyz, sel, K, axis, out,
                                                                dist2);
    else
        afps_knn_kernel<2><<<grid, 32 * kKnnWarps, 0, stream>>>(d_descs, xyz, sel, K, axis, out,
                                                                dist2);
    return cudaGetLastError();
}

}  // namespace afps
