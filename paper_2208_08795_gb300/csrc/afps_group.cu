// afps_group.cu -- ball query: the grouping step that follows sampling in a
// PointNet++ set abstraction (the paper's target, Sec. I-II).
//
// For each centroid: the first K points in storage order whose squared
// distance (dx*dx + dy*dy) + dz*dz (fp32, every operation rounded on its own)
// is below radius*radius, the remaining slots repeating the first one found.
// One warp per centroid scans 32 points per step; a ballot of the hits gives
// each hit its rank, so the first K are kept in storage order.
//
// Dimensional locality (Sec. III-A) shortens the scan: on a cloud sorted
// ascending along `axis`, the hits lie in an index range around the
// centroid's own index.  The rounded difference along the axis is monotone in
// the coordinate and a point with difference <= -r or >= r cannot be a hit
// (its square alone reaches r*r), so the warp walks 32-point chunks down
// from the centroid to the first point not excluded on the left, and stops
// the forward scan at the first chunk holding a point past the right edge.
// The result equals the full scan's exactly.
#include "afps_device.cuh"

namespace afps {

constexpr int kGroupWarps = 8;

__global__ void __launch_bounds__(32 * kGroupWarps) afps_ball_query_kernel(
    const GroupDesc* __restrict__ descs, const float* __restrict__ xyz,
    const int32_t* __restrict__ sel, float radius, int K, int axis,
    int32_t* __restrict__ out) {
    const GroupDesc d = descs[blockIdx.y];
    const int lane = threadIdx.x & 31;
    const int s = blockIdx.x * kGroupWarps + (threadIdx.x >> 5);
    if (s >= d.c) return;  // warp-uniform
    const unsigned lt = (1u << lane) - 1u;
    const float* P = xyz + 3 * d.pt_off;
    const int n = d.n;
    const int ci = min(max(sel[d.sel_off + s], 0), n - 1);
    const float cx = P[3 * ci], cy = P[3 * ci + 1], cz = P[3 * ci + 2];
    const float ca = axis == 0 ? cx : axis == 1 ? cy : cz;
    const float r2 = __fmul_rn(radius, radius);
    int32_t* row = out + (d.sel_off + s) * (int64_t)K;

    int lo = 0;
    if (axis >= 0) {
        int j0 = ci & ~31;
        while (j0 > 0) {
            const int j = j0 - 32 + lane;
            const bool left = __fsub_rn(P[3 * j + axis], ca) <= -radius;
            const unsigned b = __ballot_sync(dev::kFull, left);
            if (b) {
                lo = j0 - 32 + (31 - __clz(b)) + 1;
                break;
            }
            j0 -= 32;
        }
    }

    int cnt = 0, first = -1;
    for (int j0 = lo; j0 < n && cnt < K; j0 += 32) {
        const int j = j0 + lane;
        const bool valid = j < n;
        float px = 0.f, py = 0.f, pz = 0.f;
        if (valid) {
            px = P[3 * j];
            py = P[3 * j + 1];
            pz = P[3 * j + 2];
        }
        const bool in = valid && dev::sqdist(px, py, pz, cx, cy, cz) < r2;
        const unsigned b = __ballot_sync(dev::kFull, in);
        if (in) {
            const int q = cnt + __popc(b & lt);
            if (q < K) row[q] = j;
        }
        if (first < 0 && b) first = j0 + __ffs(b) - 1;
        cnt += __popc(b);
        if (axis >= 0) {
            const float pa = axis == 0 ? px : axis == 1 ? py : pz;
            if (__ballot_sync(dev::kFull, valid && __fsub_rn(pa, ca) >= radius)) break;
        }
    }
    for (int q = min(cnt, K) + lane; q < K; q += 32) row[q] = first;
}

cudaError_t launch_ball_query(const GroupDesc* d_descs, int32_t B, int32_t max_c,
                              const float* xyz, const int32_t* sel, float radius, int32_t K,
                              int32_t axis, int32_t* out, cudaStream_t stream) {
    if (B < 1 || max_c < 1) return cudaSuccess;
    const dim3 grid((unsigned)((max_c + kGroupWarps - 1) / kGroupWarps), (unsigned)B);
    afps_ball_query_kernel<<<grid, 32 * kGroupWarps, 0, stream>>>(d_descs, xyz, sel, radius, K,
                                                                  axis, out);
    return cudaGetLastError();
}

}  // namespace afps
