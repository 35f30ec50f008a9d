// afps_coverage.cu -- coverage radius of sample sets, on the device.
//
// The coverage radius R(S) = max_j min_{s in S} |p_j - p_s| is the quantity
// FPS greedily shrinks (property P1, Sec. II-B); it scores a sample set
// without a trained network, which lets the sampling variants be compared on
// synthetic clouds.  Squared distances are computed in fp64 from the fp32
// points, (dx*dx + dy*dy) + dz*dz with every operation rounded on its own, so
// the result can be reproduced exactly on any IEEE host.
//
// Grid (point blocks, clouds): each thread keeps the running minimum for one
// point over the cloud's samples, staged 1024 at a time in shared memory; the
// block maximum goes to the cloud's slot by an atomic max on the bits of the
// non-negative double (ordered like the values); a second launch takes the
// square roots.
#include "afps_device.cuh"

namespace afps {

constexpr int kCovThreads = 256;
constexpr int kCovTile = 1024;

__global__ void __launch_bounds__(kCovThreads) afps_coverage_kernel(
    const CoverageDesc* __restrict__ descs, const float* __restrict__ xyz,
    const int32_t* __restrict__ sel, unsigned long long* __restrict__ max_bits) {
    __shared__ double sx[kCovTile], sy[kCovTile], sz[kCovTile];
    __shared__ double warp_max[kCovThreads / 32];
    const CoverageDesc d = descs[blockIdx.y];
    const int j = blockIdx.x * kCovThreads + threadIdx.x;
    if (blockIdx.x * kCovThreads >= d.n) return;  // block-uniform
    const bool valid = j < d.n;
    double px = 0, py = 0, pz = 0;
    if (valid) {
        const float* p = xyz + 3 * (d.pt_off + j);
        px = p[0];
        py = p[1];
        pz = p[2];
    }
    double best = __longlong_as_double(0x7ff0000000000000ll);  // +inf
    for (int t0 = 0; t0 < d.c; t0 += kCovTile) {
        const int tn = min(kCovTile, d.c - t0);
        __syncthreads();
        for (int u = threadIdx.x; u < tn; u += kCovThreads) {
            const int q = min(max(sel[d.sel_off + t0 + u], 0), d.n - 1);  // stay in the cloud
            const float* s = xyz + 3 * (d.pt_off + q);
            sx[u] = s[0];
            sy[u] = s[1];
            sz[u] = s[2];
        }
        __syncthreads();
        for (int u = 0; u < tn; ++u) {
            const double dx = __dsub_rn(px, sx[u]);
            const double dy = __dsub_rn(py, sy[u]);
            const double dz = __dsub_rn(pz, sz[u]);
            const double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)),
                                        __dmul_rn(dz, dz));
            best = dd < best ? dd : best;
        }
    }
    double v = valid ? best : 0.0;
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(dev::kFull, v, o));
    if ((threadIdx.x & 31) == 0) warp_max[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = warp_max[0];
        for (int w = 1; w < kCovThreads / 32; ++w) m = fmax(m, warp_max[w]);
        atomicMax(&max_bits[blockIdx.y], (unsigned long long)__double_as_longlong(m));
    }
}

__global__ void afps_coverage_finish(const unsigned long long* __restrict__ max_bits, int32_t B,
                                     double* __restrict__ radius) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b < B) radius[b] = sqrt(__longlong_as_double((long long)max_bits[b]));
}

cudaError_t launch_coverage(const CoverageDesc* d_descs, int32_t B, int32_t max_n,
                            const float* xyz, const int32_t* sel,
                            unsigned long long* max_bits, double* radius,
                            cudaStream_t stream) {
    if (B < 1) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(max_bits, 0, sizeof(unsigned long long) * B, stream);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((max_n + kCovThreads - 1) / kCovThreads), (unsigned)B);
    afps_coverage_kernel<<<grid, kCovThreads, 0, stream>>>(d_descs, xyz, sel, max_bits);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    afps_coverage_finish<<<(B + 127) / 128, 128, 0, stream>>>(max_bits, B, radius);
    return cudaGetLastError();
}

}  // namespace afps
