// 2-D implicit-step operators (JAX-PF Eq. 13-14 on a 2-D Q1 mesh) with the
// double well f = W u^2 (1-u)^2, r the gradient and H the Hessian of
// E_h = sum_e sum_q w|J| [f(U_q) + kappa/2 |grad U_q|^2]:
//   Allen-Cahn:  R(U) = M (U - U^n)/dt + L r(U),     J v = M v / dt + L H(U) v
//   split Cahn-Hilliard (Eq. 9-10), unknowns [c; mu]:
//                R = [M (c - c^n)/dt + K_M mu;  M mu - r(c)]
//                J [v_c; v_mu] = [M v_c / dt + K_M v_mu;  M v_mu - H(c) v_c]
// As in 3-D all are evaluated scaled by the lumped mass (M^-1 R, M^-1 J v) on
// a tile with mirror images beyond the mesh, where every node uses the
// interior formula; an optional final multiplication by m_i gives R and J v
// themselves.
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

// Mirror image of node index k on an axis of n nodes (period 2(n-1)).  Halo
// indices lie within one period of the axis, where a reflection at each end
// gives the image without the integer division.
__device__ __forceinline__ int mirror(int k, int n) {
  const int p = 2 * (n - 1);
  if (k >= 1 - n && k <= p) return k < 0 ? -k : (k < n ? k : p - k);
  k %= p;
  if (k < 0) k += p;
  return k < n ? k : p - k;
}

__device__ __forceinline__ float gpt(int i) { return i ? kGHi : kGLo; }

// 9-point stencil s at node (y, x) of a staged plane.  The Q1 stiffness rows
// sum to zero (c0 = -2 cx - 2 cy - 4 cd), so K v is applied to the differences
// v_j - v_i: for smooth fields each difference of neighbouring FP32 values is
// exact, where c0 v_i + sum c_j v_j would cancel to a few significant bits.
template <int W_>
__device__ __forceinline__ float stencil(const float (*V)[W_], int y, int x, const Stencil2D& k) {
  const float c = V[y][x];
  return k.cx * ((V[y][x - 1] - c) + (V[y][x + 1] - c)) +
         k.cy * ((V[y - 1][x] - c) + (V[y + 1][x] - c)) +
         k.cd * (((V[y - 1][x - 1] - c) + (V[y - 1][x + 1] - c)) +
                 ((V[y + 1][x - 1] - c) + (V[y + 1][x + 1] - c)));
}

template <bool kJVP, bool kCH>
__global__ void __launch_bounds__(kThreads) k_implicit2d(const Implicit2DArgs a) {
  // sU: U (AC) or c; sW: U^n / v (AC) or c^n / v_c; sM (CH): mu (residual) or v_mu (JVP)
  __shared__ float sU[SY][SX], sW[SY][SX], sM[kCH ? SY : 1][kCH ? SX : 1];
  __shared__ float sE[4][EY][EX];
  const int tiles_x = (a.nx + TX - 1) / TX;
  const int x0 = (blockIdx.x % tiles_x) * TX, y0 = (blockIdx.x / tiles_x) * TY;
  const int64_t N = (int64_t)a.nx * a.ny;

  for (int i = threadIdx.x; i < SX * SY; i += kThreads) {
    const int lx = i % SX, ly = i / SX;
    const int64_t g = (int64_t)mirror(y0 - 1 + ly, a.ny) * a.nx + mirror(x0 - 1 + lx, a.nx);
    sU[ly][lx] = a.U[g];
    sW[ly][lx] = a.W[g];
    if (kCH) sM[ly][lx] = kJVP ? a.W[N + g] : a.U[N + g];
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
    const float ks = stencil(V, y, x, a.k);
    const float own = kJVP ? sW[y][x] : (sU[y][x] - sW[y][x]);
    float wm = 1.0f;
    if (a.unscaled) {
      const float wx = (gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f;
      const float wy = (gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f;
      wm = a.cell * wx * wy;
    }
    const int64_t o = (int64_t)gy * a.nx + gx;
    if (kCH) {
      // c row: own / dt + M_c m^-1 K (mu or v_mu);  mu row: (mu or v_mu) - m^-1 (r or H v_c)
      a.out[o] = wm * fmaf(own, a.inv_dt, stencil(sM, y, x, a.km));
      a.out[N + o] = wm * (sM[y][x] - (acc + ks));
    } else {
      a.out[o] = wm * fmaf(own, a.inv_dt, a.mob * (acc + ks));
    }
  }
}

}  // namespace

cudaError_t launch_residual2d(const Implicit2DArgs& a, cudaStream_t s) {
  const int tiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
  if (a.ch)
    k_implicit2d<false, true><<<tiles, kThreads, 0, s>>>(a);
  else
    k_implicit2d<false, false><<<tiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_jvp2d(const Implicit2DArgs& a, cudaStream_t s) {
  const int tiles = ((a.nx + TX - 1) / TX) * ((a.ny + TY - 1) / TY);
  if (a.ch)
    k_implicit2d<true, true><<<tiles, kThreads, 0, s>>>(a);
  else
    k_implicit2d<true, false><<<tiles, kThreads, 0, s>>>(a);
  return cudaGetLastError();
}

}  // namespace pf
