// Plain two-pass explicit step on a 2-D mesh: the comparison form for the
// fused kernel (same discretisation, Eq. 11-12 and the split form of Eq. 9-10;
// same shifted FP32 state d = u - shift and the same constants).
//
// It is what a direct node-centric implementation does: one thread per node
// gathers its (up to) four elements, evaluates u and f'(u) at each element's
// 2x2 Gauss points, weights them with the node's shape function, and applies
// the 9-point Q1 stiffness stencil; boundaries reflect the indices (the mirror
// extension of the zero-flux operators).  For Cahn-Hilliard the chemical
// potential mu makes a round trip through HBM between two launches:
//   pass 1: mu = sum_q N_i(q) f'(u_q) / 4 + kappa/m K d       (written)
//   pass 2: d' = d - dt M/m K mu                               (mu read back)
// Allen-Cahn is one pass.  No ghost frame, no register sweep, no graph.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kBX = 32, kBY = 8;

__device__ __forceinline__ int refl(int i, int n) { return i < 0 ? -i : (i >= n ? 2 * n - 2 - i : i); }

__device__ __forceinline__ float at(const float* __restrict__ p, int i, int j, int nx, int ny) {
  return p[(int64_t)refl(j, ny) * nx + refl(i, nx)];
}

// 9-point stencil s applied to p at node (i, j)
__device__ __forceinline__ float stencil(const float* __restrict__ p, int i, int j, int nx, int ny,
                                         const Stencil2D& s) {
  const float c = at(p, i, j, nx, ny);
  const float x = at(p, i - 1, j, nx, ny) + at(p, i + 1, j, nx, ny);
  const float y = at(p, i, j - 1, nx, ny) + at(p, i, j + 1, nx, ny);
  const float d = at(p, i - 1, j - 1, nx, ny) + at(p, i + 1, j - 1, nx, ny) +
                  at(p, i - 1, j + 1, nx, ny) + at(p, i + 1, j + 1, nx, ny);
  return s.c0 * c + s.cx * x + s.cy * y + s.cd * d;
}

// sum over the node's elements and their Gauss points of N_i(q) * P(u_q), with
// P(d) = p0 + d (p1 + d (p2 + d p3)) = f'(shift + d) / 4 times the stage factor
__device__ float fprime_quad(const float* __restrict__ p, int i, int j, int nx, int ny,
                             const Explicit2DArgs& a) {
  const float g[2] = {0.5f - 0.28867513459481287f, 0.5f + 0.28867513459481287f};
  float acc = 0.0f;
#pragma unroll
  for (int ey = 0; ey < 2; ++ey)
#pragma unroll
    for (int ex = 0; ex < 2; ++ex) {
      // element with corners (i-1+ex .. i+ex, j-1+ey .. j+ey); the node is its
      // local corner (1 - ex, 1 - ey)
      const int x0 = i - 1 + ex, y0 = j - 1 + ey;
      const float u00 = at(p, x0, y0, nx, ny), u10 = at(p, x0 + 1, y0, nx, ny);
      const float u01 = at(p, x0, y0 + 1, nx, ny), u11 = at(p, x0 + 1, y0 + 1, nx, ny);
#pragma unroll
      for (int qy = 0; qy < 2; ++qy)
#pragma unroll
        for (int qx = 0; qx < 2; ++qx) {
          const float sx = g[qx], sy = g[qy];
          const float u = (1 - sy) * ((1 - sx) * u00 + sx * u10) + sy * ((1 - sx) * u01 + sx * u11);
          const float nxw = ex ? (1 - sx) : sx;  // local x of the node is 1 - ex
          const float nyw = ey ? (1 - sy) : sy;
          acc += nxw * nyw * (a.p0 + u * (a.p1 + u * (a.p2 + u * a.p3)));
        }
    }
  return acc;
}

__global__ void __launch_bounds__(kBX* kBY) k_plain_mu(const float* __restrict__ d, Explicit2DArgs a,
                                                      float* __restrict__ mu) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = block_row() * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  mu[(int64_t)j * a.nx + i] = fprime_quad(d, i, j, a.nx, a.ny, a) + stencil(d, i, j, a.nx, a.ny, a.k1);
}

__global__ void __launch_bounds__(kBX* kBY) k_plain_c(const float* __restrict__ d,
                                                     const float* __restrict__ mu, Explicit2DArgs a,
                                                     float* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = block_row() * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const int64_t k = (int64_t)j * a.nx + i;
  out[k] = d[k] + stencil(mu, i, j, a.nx, a.ny, a.k2);
}

__global__ void __launch_bounds__(kBX* kBY) k_plain_ac(const float* __restrict__ d, Explicit2DArgs a,
                                                      float* __restrict__ out) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = block_row() * kBY + threadIdx.y;
  if (i >= a.nx || j >= a.ny) return;
  const int64_t k = (int64_t)j * a.nx + i;
  out[k] = d[k] + fprime_quad(d, i, j, a.nx, a.ny, a) + stencil(d, i, j, a.nx, a.ny, a.k1);
}

}  // namespace

cudaError_t launch_plain2d(bool ch, const Explicit2DArgs& a, const float* d, float* mu, float* out,
                           cudaStream_t s) {
  const dim3 blk(kBX, kBY), grd = row_grid((a.nx + kBX - 1) / kBX, (a.ny + kBY - 1) / kBY);
  if (ch) {
    k_plain_mu<<<grd, blk, 0, s>>>(d, a, mu);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_plain_c<<<grd, blk, 0, s>>>(d, mu, a, out);
  } else {
    k_plain_ac<<<grd, blk, 0, s>>>(d, a, out);
  }
  return cudaGetLastError();
}

}  // namespace pf
