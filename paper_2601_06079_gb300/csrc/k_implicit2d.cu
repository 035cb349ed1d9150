// 2-D implicit-step operators for the Allen-Cahn double well (JAX-PF
// Eq. 13-14 on a 2-D Q1 mesh):
//   R(U) = M (U - U^n)/dt + L r(U),     J v = M v / dt + L H(U) v,
// r the gradient and H the Hessian of E_h = sum_e sum_q w|J| [f(U_q) +
// kappa/2 |grad U_q|^2], f = W u^2 (1-u)^2.  As in 3-D both are evaluated
// scaled by the lumped mass (G = M^-1 R, M^-1 J v) on a tile with mirror
// images beyond the mesh, where every node uses the interior formula; an
// optional final multiplication by m_i gives R and J v themselves.
//
// One block per 32 x 16 node tile: U and v (or U^n) are staged with a 1-node
// halo; every element touching the tile evaluates f'(u_q) (residual) or
// f''(u_q) v_q (JVP) at its 2x2 Gauss points and projects it to its corners;
// a node-centric gather of the 4 element contributions plus the assembled
// 9-point stiffness stencil gives the output.  No atomics.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int TX = 32, TY = 16;            // output tile
constexpr int kThreads = 256;
constexpr int SX = TX + 2, SY = TY + 2;    // nodes with a 1-node halo
constexpr int EX = TX + 1, EY = TY + 1;    // elements touching the tile nodes

__device__ __forceinline__ int mirror(int k, int n) {
  const int p = 2 * (n - 1);
  k %= p;
  if (k < 0) k += p;
  return k < n ? k : p - k;
}

__device__ __forceinline__ float gpt(int i) { return i ? kGHi : kGLo; }

template <bool kJVP>
__global__ void __launch_bounds__(kThreads) k_implicit2d(const Implicit2DArgs a) {
  __shared__ float sU[SY][SX], sW[SY][SX];
  __shared__ float sE[4][EY][EX];
  const int tiles_x = (a.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;

  for (int i = threadIdx.x; i < SX * SY; i += kThreads) {
    const int lx = i % SX, ly = i / SX;
    const int64_t g = (int64_t)mirror(y0 - 1 + ly, a.ny) * a.nx + mirror(x0 - 1 + lx, a.nx);
    sU[ly][lx] = a.U[g];
    sW[ly][lx] = a.W[g];
  }
  __syncthreads();

  // element (ey, ex) has lower-left node (ey, ex) in halo coordinates
  for (int i = threadIdx.x; i < EX * EY; i += kThreads) {
    const int ex = i % EX, ey = i / EX;
    const float u[4] = {sU[ey][ex], sU[ey][ex + 1], sU[ey + 1][ex], sU[ey + 1][ex + 1]};
    const float v[4] = {sW[ey][ex], sW[ey][ex + 1], sW[ey + 1][ex], sW[ey + 1][ex + 1]};
    float t[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float xi = gpt(q & 1), et = gpt(q >> 1);
      const float ub = fmaf(xi, u[1] - u[0], u[0]), ut = fmaf(xi, u[3] - u[2], u[2]);
      const float uq = fmaf(et, ut - ub, ub);
      if (kJVP) {
        const float vb = fmaf(xi, v[1] - v[0], v[0]), vt = fmaf(xi, v[3] - v[2], v[2]);
        const float vq = fmaf(et, vt - vb, vb);
        // f''(u) = 2W (1 - 6u + 6u^2)
        t[q] = a.dw2 * fmaf(6.0f * uq, uq - 1.0f, 1.0f) * vq;
      } else {
        // f'(u) = 2W u (1-u)(1-2u)
        t[q] = a.dw2 * uq * (1.0f - uq) * (1.0f - 2.0f * uq);
      }
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      float s = 0.0f;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float xi = gpt(q & 1), et = gpt(q >> 1);
        s = fmaf(t[q], ((c & 1) ? xi : 1.0f - xi) * ((c >> 1) ? et : 1.0f - et), s);
      }
      sE[c][ey][ex] = 0.25f * s;  // Gauss weight |cell|/4 over the interior mass |cell|
    }
  }
  __syncthreads();

  for (int i = threadIdx.x; i < TX * TY; i += kThreads) {
    const int lx = i % TX, ly = i / TX;
    const int gx = x0 + lx, gy = y0 + ly;
    if (gx >= a.nx || gy >= a.ny) continue;
    const int x = lx + 1, y = ly + 1;
    const float acc = sE[0][y][x] + sE[1][y][x - 1] + sE[2][y - 1][x] + sE[3][y - 1][x - 1];
    const float (*V)[SX] = kJVP ? sW : sU;  // the stiffness acts on v (JVP) or U (residual)
    const Stencil2D& k = a.k;
    const float ks = k.c0 * V[y][x] + k.cx * (V[y][x - 1] + V[y][x + 1]) +
                     k.cy * (V[y - 1][x] + V[y + 1][x]) +
                     k.cd * (V[y - 1][x - 1] + V[y - 1][x + 1] + V[y + 1][x - 1] + V[y + 1][x + 1]);
    const float own = kJVP ? sW[y][x] : (sU[y][x] - sW[y][x]);
    float g = fmaf(own, a.inv_dt, a.mob * (acc + ks));
    if (a.unscaled) {
      const float wx = (gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f;
      const float wy = (gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f;
      g *= a.cell * wx * wy;
    }
    a.out[(int64_t)gy * a.nx + gx] = g;
  }
}

}  // namespace

cudaError_t launch_residual2d(const Implicit2DArgs& a, cudaStream_t s) {
  const int tiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
  k_implicit2d<false><<<tiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_jvp2d(const Implicit2DArgs& a, cudaStream_t s) {
  const int tiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
  k_implicit2d<true><<<tiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pf
