// 3-D implicit-step operators for n_f order parameters (Fan-Chen grain growth
// or the double well), JAX-PF Eq. 13-14:
//   R(U) = M (U - U^n)/dt + L r(U),     J v = M v / dt + L H(U) v,
// with r the gradient and H the Hessian of E_h = sum_e sum_q w|J| [f(U_q) +
// kappa/2 |grad U_q|^2].  Both are evaluated scaled by the lumped mass,
// G = M^-1 R and M^-1 J v, on a mirror-extended tile: the mirror images of
// boundary elements double the partial sums exactly where the lumped mass
// halves, so every node uses the interior formula (an optional final
// multiplication by m_i gives R and J v themselves).
//
// Work split: one block per 8x8x8 node tile.  The block stages U (and v, or
// U^n) for the 10^3 nodes around it in shared memory, mirrored at the mesh
// boundary, then evaluates all 9^3 elements touching the tile:
//   phase 1: per element and Gauss point, S2 = sum_f U_f^2 (and T =
//            sum_f U_f v_f for the JVP), the only couplings between fields;
//   phase 2: per field, the Gauss values (trilinear, sum-factorised), the
//            pointwise f' or H v, the weights back to the 8 corners into a
//            per-element buffer, then a node-centric gather of the 8 element
//            contributions plus the assembled 27-point stiffness stencil.
// No atomics: the gather order is fixed, so results are bitwise repeatable.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kT = 8;                 // output nodes per tile edge
constexpr int kN = kT + 2;            // staged nodes per edge (1 halo each side)
constexpr int kE = kT + 1;            // elements per edge touching the tile
constexpr int kNodes = kN * kN * kN;  // 1000
constexpr int kElems = kE * kE * kE;  // 729
#ifndef PF_IMP_THREADS
#define PF_IMP_THREADS 1024
#endif
constexpr int kThreads = PF_IMP_THREADS;

__device__ __forceinline__ int mirror(int k, int n) {
  const int p = 2 * (n - 1);
  k %= p;
  if (k < 0) k += p;
  return k < n ? k : p - k;
}

// values at the two Gauss points of a segment from its end values
__device__ __forceinline__ void interp1(float a, float b, float& lo, float& hi) {
  const float d = b - a;
  lo = fmaf(kGLo, d, a);
  hi = fmaf(kGHi, d, a);
}

// weights back: contributions of the two Gauss values to the segment's ends
__device__ __forceinline__ void project1(float lo, float hi, float& a, float& b) {
  const float d = hi - lo;
  a = fmaf(kGLo, d, lo);      // g_hi lo + g_lo hi
  b = fmaf(-kGLo, d, hi);     // g_lo lo + g_hi hi
}

// 8 corner values c[z][y][x] -> 8 Gauss values q[z][y][x] (tensor product)
__device__ __forceinline__ void interp3(const float c[8], float q[8]) {
  float t[8], u[8];
#pragma unroll
  for (int zy = 0; zy < 4; ++zy) interp1(c[2 * zy], c[2 * zy + 1], t[2 * zy], t[2 * zy + 1]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) interp1(t[4 * z + x], t[4 * z + 2 + x], u[4 * z + x], u[4 * z + 2 + x]);
#pragma unroll
  for (int yx = 0; yx < 4; ++yx) interp1(u[yx], u[4 + yx], q[yx], q[4 + yx]);
}

// transpose of interp3: Gauss values -> corner contributions
__device__ __forceinline__ void project3(const float q[8], float c[8]) {
  float t[8], u[8];
#pragma unroll
  for (int yx = 0; yx < 4; ++yx) project1(q[yx], q[4 + yx], t[yx], t[4 + yx]);
#pragma unroll
  for (int z = 0; z < 2; ++z)
#pragma unroll
    for (int x = 0; x < 2; ++x) project1(t[4 * z + x], t[4 * z + 2 + x], u[4 * z + x], u[4 * z + 2 + x]);
#pragma unroll
  for (int zy = 0; zy < 4; ++zy) project1(u[2 * zy], u[2 * zy + 1], c[2 * zy], c[2 * zy + 1]);
}

__device__ __forceinline__ int nidx(int x, int y, int z) { return (z * kN + y) * kN + x; }

template <int NF, bool kJVP>
__global__ void __launch_bounds__(kThreads) k_implicit3d(const Implicit3DArgs a) {
  extern __shared__ float smem[];
  float* sU = smem;                          // [NF][kNodes]
  float* sW = sU + NF * kNodes;              // v (JVP) or U^n (residual)
  // per-element values are stored [8][kElems] (Gauss point or corner major), so
  // that consecutive threads (consecutive elements) hit consecutive banks
  float* sS = sW + NF * kNodes;              // [8][kElems] S2 at Gauss points
  float* sTq = sS + kElems * 8;              // [8][kElems] T (JVP only)
  float* sE = sTq + (kJVP ? kElems * 8 : 0); // [8][kElems] corner contributions of one field

  const int tiles_x = (a.nx + kT - 1) / kT, tiles_y = (a.ny + kT - 1) / kT;
  const int tile = blockIdx.x;
  const int x0 = (tile % tiles_x) * kT, y0 = ((tile / tiles_x) % tiles_y) * kT,
            z0 = (tile / (tiles_x * tiles_y)) * kT;
  const int64_t N = (int64_t)a.nx * a.ny * a.nz;

  // stage U and v / U^n with mirror images beyond the mesh
  for (int i = threadIdx.x; i < kNodes; i += kThreads) {
    const int lx = i % kN, ly = (i / kN) % kN, lz = i / (kN * kN);
    const int gx = mirror(x0 - 1 + lx, a.nx), gy = mirror(y0 - 1 + ly, a.ny),
              gz = mirror(z0 - 1 + lz, a.nz);
    const int64_t g = ((int64_t)gz * a.ny + gy) * a.nx + gx;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      sU[f * kNodes + i] = a.U[f * N + g];
      sW[f * kNodes + i] = a.W[f * N + g];
    }
  }
  __syncthreads();

  // phase 1: field couplings at the Gauss points of every element
  for (int e = threadIdx.x; e < kElems; e += kThreads) {
    const int ex = e % kE, ey = (e / kE) % kE, ez = e / (kE * kE);
    const int base = nidx(ex, ey, ez);
    float S2[8], T[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) S2[q] = T[q] = 0.0f;
#pragma unroll
    for (int f = 0; f < NF; ++f) {
      float c[8], uq[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        c[k] = sU[f * kNodes + base + ((k >> 2) * kN + ((k >> 1) & 1)) * kN + (k & 1)];
      interp3(c, uq);
      if (kJVP) {
        float vq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          c[k] = sW[f * kNodes + base + ((k >> 2) * kN + ((k >> 1) & 1)) * kN + (k & 1)];
        interp3(c, vq);
#pragma unroll
        for (int q = 0; q < 8; ++q) T[q] = fmaf(uq[q], vq[q], T[q]);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) S2[q] = fmaf(uq[q], uq[q], S2[q]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      sS[q * kElems + e] = S2[q];
      if (kJVP) sTq[q * kElems + e] = T[q];
    }
  }
  __syncthreads();

  // phase 2: one field at a time
  for (int f = 0; f < NF; ++f) {
    const float* Uf = sU + f * kNodes;
    const float* Wf = sW + f * kNodes;
    for (int e = threadIdx.x; e < kElems; e += kThreads) {
      const int ex = e % kE, ey = (e / kE) % kE, ez = e / (kE * kE);
      const int base = nidx(ex, ey, ez);
      float c[8], uq[8], vq[8], hq[8], out[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) c[k] = Uf[base + ((k >> 2) * kN + ((k >> 1) & 1)) * kN + (k & 1)];
      interp3(c, uq);
      if (kJVP) {
#pragma unroll
        for (int k = 0; k < 8; ++k)
          c[k] = Wf[base + ((k >> 2) * kN + ((k >> 1) & 1)) * kN + (k & 1)];
        interp3(c, vq);
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const float u = uq[q], s2 = sS[q * kElems + e];
        if (a.double_well) {
          // f = W u^2 (1-u)^2:  f' = 2W u (1-u)(1-2u),  f'' = 2W (1 - 6u + 6u^2)
          hq[q] = kJVP ? a.dw2 * fmaf(6.0f * u, u - 1.0f, 1.0f) * vq[q]
                       : a.dw2 * u * (1.0f - u) * (1.0f - 2.0f * u);
        } else {
          // Fan-Chen: f'_f = u (-a + 2g S2 + (b - 2g) u^2)
          //           (H v)_f = (-a + 2g S2 + (3b - 6g) u^2) v_f + 4g u T
          const float base_c = fmaf(a.two_gamma, s2, -a.alpha);
          hq[q] = kJVP ? fmaf(fmaf(a.c3b6g, u * u, base_c), vq[q],
                              a.four_gamma * u * sTq[q * kElems + e])
                       : u * fmaf(a.cb2g, u * u, base_c);
        }
      }
      project3(hq, out);
#pragma unroll
      for (int k = 0; k < 8; ++k) sE[k * kElems + e] = out[k];
    }
    __syncthreads();
    // node gather: 8 elements around the node, stiffness stencil, mass term
    for (int i = threadIdx.x; i < kT * kT * kT; i += kThreads) {
      const int lx = 1 + i % kT, ly = 1 + (i / kT) % kT, lz = 1 + i / (kT * kT);
      const int gx = x0 + lx - 1, gy = y0 + ly - 1, gz = z0 + lz - 1;
      if (gx >= a.nx || gy >= a.ny || gz >= a.nz) continue;
      float acc = 0.0f;
#pragma unroll
      for (int k = 0; k < 8; ++k) {  // element with corner k at this node
        const int ex = lx - (k & 1), ey = ly - ((k >> 1) & 1), ez = lz - (k >> 2);
        acc += sE[k * kElems + (ez * kE + ey) * kE + ex];
      }
      const float* V = kJVP ? Wf : Uf;  // the stiffness acts on v (JVP) or U (residual)
      const int c0 = nidx(lx, ly, lz);
      float ks = a.kc[0] * V[c0];
#pragma unroll
      for (int dz = -1; dz <= 1; ++dz)
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
          for (int dx = -1; dx <= 1; ++dx) {
            const int cls = (dx != 0) + 2 * (dy != 0) + 4 * (dz != 0);
            if (cls == 0) continue;
            ks = fmaf(a.kc[cls], V[c0 + (dz * kN + dy) * kN + dx], ks);
          }
      // G = (u - u^n)/dt + L (F/m + kappa K u / m)   or   v/dt + L (H v / m + kappa K v / m)
      const float own = kJVP ? Wf[c0] : (Uf[c0] - Wf[c0]);
      float g = fmaf(own, a.inv_dt, a.mob * (0.125f * acc + ks));
      if (a.unscaled) {
        const float wx = (gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f;
        const float wy = (gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f;
        const float wz = (gz == 0 || gz == a.nz - 1) ? 0.5f : 1.0f;
        g *= a.cell * wx * wy * wz;
      }
      a.out[f * N + ((int64_t)gz * a.ny + gy) * a.nx + gx] = g;
    }
    __syncthreads();
  }
}

template <int NF, bool kJVP>
cudaError_t launch_nf(const Implicit3DArgs& a, cudaStream_t s) {
  const size_t smem =
      sizeof(float) * (2 * NF * kNodes + kElems * 8 * (kJVP ? 3 : 2));
  static bool configured[2] = {false, false};
  if (!configured[kJVP]) {
    cudaError_t e = cudaFuncSetAttribute(k_implicit3d<NF, kJVP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured[kJVP] = true;
  }
  const int tiles = ((a.nx + kT - 1) / kT) * ((a.ny + kT - 1) / kT) * ((a.nz + kT - 1) / kT);
  k_implicit3d<NF, kJVP><<<tiles, kThreads, smem, s>>>(a);
  return cudaGetLastError();
}

template <bool kJVP>
cudaError_t launch_any(const Implicit3DArgs& a, cudaStream_t s) {
  switch (a.nf) {
    case 1: return launch_nf<1, kJVP>(a, s);
    case 2: return launch_nf<2, kJVP>(a, s);
    case 3: return launch_nf<3, kJVP>(a, s);
    case 4: return launch_nf<4, kJVP>(a, s);
    case 5: return launch_nf<5, kJVP>(a, s);
    case 6: return launch_nf<6, kJVP>(a, s);
    case 7: return launch_nf<7, kJVP>(a, s);
    case 8: return launch_nf<8, kJVP>(a, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace

cudaError_t launch_residual3d(const Implicit3DArgs& a, cudaStream_t s) {
  return launch_any<false>(a, s);
}

cudaError_t launch_jvp3d(const Implicit3DArgs& a, cudaStream_t s) { return launch_any<true>(a, s); }

}  // namespace pf
