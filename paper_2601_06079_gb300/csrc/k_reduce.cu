// FP64 diagnostics: discrete free energy E_h (JAX-PF Eq. 5-6 with the 2x2
// Gauss rule) and the mass integral sum_i m_i u_i with the lumped mass.
// Per-element values are formed in FP32 from the shifted state and summed
// in FP64: warp shuffles, then shared memory, one partial per block, then a
// single-block pass over the partials in a fixed order, so the result does
// not depend on scheduling (no atomics).
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kThreads = 256;
constexpr int kMaxBlocks = 1024;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum of two values; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[kThreads / 32], sb[kThreads / 32];
  a = warp_sum(a);
  b = warp_sum(b);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) {
    sa[w] = a;
    sb[w] = b;
  }
  __syncthreads();
  if (w == 0) {
    a = (l < kThreads / 32) ? sa[l] : 0.0;
    b = (l < kThreads / 32) ? sb[l] : 0.0;
    a = warp_sum(a);
    b = warp_sum(b);
  }
}

__device__ __forceinline__ float quartic(float d, const Energy2DArgs& a) {
  return fmaf(fmaf(fmaf(fmaf(a.q4, d, a.q3), d, a.q2), d, a.q1), d, a.q0);
}

__global__ void __launch_bounds__(kThreads) k_energy2d(const Energy2DArgs a, double* partials) {
  const int64_t n = (int64_t)a.nx * a.ny;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  const float ihx = (float)(1.0 / a.hx), ihy = (float)(1.0 / a.hy);
  const double cell = a.hx * a.hy;
  double e = 0.0, m = 0.0;
  for (int64_t idx = (int64_t)blockIdx.x * kThreads + threadIdx.x; idx < n; idx += stride) {
    const int i = (int)(idx % a.nx), j = (int)(idx / a.nx);
    const double wx = (i == 0 || i == a.nx - 1) ? 0.5 : 1.0;
    const double wy = (j == 0 || j == a.ny - 1) ? 0.5 : 1.0;
    const float d00 = a.d[idx];
    m += cell * wx * wy * ((double)a.shift + (double)d00);
    if (i < a.nx - 1 && j < a.ny - 1) {
      const float d10 = a.d[idx + 1], d01 = a.d[idx + a.nx], d11 = a.d[idx + a.nx + 1];
      float s = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float xi = (q & 1) ? kGHi : kGLo, eta = (q & 2) ? kGHi : kGLo;
        const float b = fmaf(xi, d10 - d00, d00);       // bottom edge at xi
        const float t = fmaf(xi, d11 - d01, d01);       // top edge at xi
        const float v = fmaf(eta, t - b, b);
        const float gx = fmaf(eta, (d11 - d01) - (d10 - d00), d10 - d00) * ihx;
        const float gy = fmaf(xi, (d11 - d10) - (d01 - d00), d01 - d00) * ihy;
        s += quartic(v, a) + 0.5f * a.kappa * fmaf(gx, gx, gy * gy);
      }
      e += 0.25 * cell * (double)s;
    }
  }
  block_sum2(e, m);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = e;
    partials[2 * blockIdx.x + 1] = m;
  }
}

__global__ void __launch_bounds__(kThreads) k_sum_partials(const double* partials, int nblocks,
                                                           double* result) {
  double e = 0.0, m = 0.0;
  for (int b = threadIdx.x; b < nblocks; b += kThreads) {
    e += partials[2 * b];
    m += partials[2 * b + 1];
  }
  block_sum2(e, m);
  if (threadIdx.x == 0) {
    result[0] = e;
    result[1] = m;
  }
}

}  // namespace

int energy2d_blocks(int nx, int ny) {
  const int64_t n = (int64_t)nx * ny;
  int64_t b = (n + kThreads - 1) / kThreads;
  return (int)(b < kMaxBlocks ? b : kMaxBlocks);
}

cudaError_t launch_energy2d(const Energy2DArgs& a, double* partials, double* result,
                            cudaStream_t s) {
  const int nb = energy2d_blocks(a.nx, a.ny);
  k_energy2d<<<nb, kThreads, 0, s>>>(a, partials);
  k_sum_partials<<<1, kThreads, 0, s>>>(partials, nb, result);
  return cudaGetLastError();
}

}  // namespace pf
