// Fused 2-D explicit step kernels: element gather -> Gauss-point values ->
// f'(u_q) -> node-centric gather of the element contributions -> gradient
// stencil -> lumped-mass Euler update (JAX-PF Eq. 11-12; Cahn-Hilliard via the
// split form of Eq. 9-10).  One pass reads the state once and writes it once.
//
// Layout and work split.  A warp owns 128 consecutive columns (4 per lane,
// one float4 per row) and sweeps down a band of rows, keeping a sliding
// window of rows in registers.  Neighbouring columns come from the adjacent
// lane by warp shuffle, so no shared memory and no block barrier is used and
// every element is evaluated exactly once per warp.  Lanes 0 and 31 are halo
// lanes (their outer columns lack a neighbour), so warps overlap by 8
// columns and each writes the 120 columns of lanes 1..30.
//
// Quadrature is sum-factorised: per row, two x-interpolated values per
// segment; per element, the four Gauss values from the segment values of its
// two rows; the weights N_a(q) are applied back the same way (y first into
// per-segment sums S, then x into the nodes).  The linear gradient term is
// the exact assembled 9-point stencil of the Q1 stiffness (2x2 Gauss
// integrates it exactly).  Zero-flux boundaries are the mirror extension
// about the boundary nodes, which equals the partial element sets divided by
// the partial lumped masses (both double when mirrored), so every node uses
// the interior formula.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kCols = 4;                      // columns per lane
constexpr int kOutCols = 32 * kCols - 2 * kCols;  // 120 output columns per warp
constexpr int kWarps = 4;                     // warps per block, stacked in y
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ int reflect(int k, int n) {
  const int p = 2 * (n - 1);
  k %= p;
  if (k < 0) k += p;
  return k < n ? k : p - k;
}

__device__ __forceinline__ void load_row(const float* __restrict__ row, int x, int nx, bool vec,
                                         float* v) {
  if (vec && x >= 0 && x + 3 < nx) {
    const float4 t = __ldg(reinterpret_cast<const float4*>(row + x));
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = __ldg(row + reflect(x + c, nx));
  }
}

__device__ __forceinline__ void store_row(float* __restrict__ row, int x, int nx, bool vec,
                                          const float* v) {
  if (vec && x + 3 < nx) {
    *reinterpret_cast<float4*>(row + x) = make_float4(v[0], v[1], v[2], v[3]);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c)
      if (x + c < nx) row[x + c] = v[c];
  }
}

__device__ __forceinline__ float cubic(float d, float p0, float p1, float p2, float p3) {
  return fmaf(fmaf(fmaf(p3, d, p2), d, p1), d, p0);
}

// Stencil at one column from three rows (own values and horizontal-neighbour sums).
__device__ __forceinline__ float stencil(const Stencil2D& k, float s_own, float s_hs, float c_own,
                                         float c_hs, float n_own, float n_hs) {
  return fmaf(k.cd, s_hs + n_hs, fmaf(k.cy, s_own + n_own, fmaf(k.cx, c_hs, k.c0 * c_own)));
}

// Horizontal neighbour sums of a row segment (own 4 values + lane neighbours).
__device__ __forceinline__ void hsum(const float* v, float left, float right, float* hs) {
  hs[0] = left + v[1];
  hs[1] = v[0] + v[2];
  hs[2] = v[1] + v[3];
  hs[3] = v[2] + right;
}

template <bool kCH, int kTY>
__global__ void __launch_bounds__(kWarps * 32) k_explicit2d(const Explicit2DArgs a) {
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  const int x = blockIdx.x * kOutCols - kCols + kCols * lane;
  const int y0 = (blockIdx.y * kWarps + warp) * kTY;
  if (y0 >= a.ny) return;  // warp-uniform
  const bool vec = a.vec_ok != 0;
  const int nx = a.nx, ny = a.ny;
  constexpr int kLag = kCH ? 2 : 1;
  constexpr int kIters = kTY + 2 * kLag;

  // sliding window (row k-1 = "1", row k-2 = "2")
  float c1[4] = {0, 0, 0, 0}, h1[4] = {0, 0, 0, 0};
  float c2[4] = {0, 0, 0, 0}, h2[4] = {0, 0, 0, 0};
  float am1[4] = {0, 0, 0, 0}, ap1[4] = {0, 0, 0, 0};  // x-interp of row k-1
  float tl1[4] = {0, 0, 0, 0}, th1[4] = {0, 0, 0, 0};  // element row k-2 -> node row k-1
  float mua[4] = {0, 0, 0, 0}, mha[4] = {0, 0, 0, 0};  // CH: mu row k-3
  float mub[4] = {0, 0, 0, 0}, mhb[4] = {0, 0, 0, 0};  // CH: mu row k-2

  float nxt[4];
  load_row(a.in + (int64_t)reflect(y0 - kLag, ny) * nx, x, nx, vec, nxt);

#pragma unroll 1
  for (int it = 0; it < kIters; ++it) {
    const int k = y0 - kLag + it;
    float c[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) c[v] = nxt[v];
    load_row(a.in + (int64_t)reflect(k + 1, ny) * nx, x, nx, vec, nxt);  // prefetch row k+1

    const float cl = __shfl_up_sync(kFull, c[3], 1);
    const float cr = __shfl_down_sync(kFull, c[0], 1);
    float hs[4];
    hsum(c, cl, cr, hs);

    // x-interpolation of row k on segments x+s .. x+s+1 at xi = g_lo (am), g_hi (ap)
    float am[4], ap[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float right = (s < 3) ? c[s + 1] : cr;
      am[s] = fmaf(kGHi, c[s], kGLo * right);
      ap[s] = fmaf(kGLo, c[s], kGHi * right);
    }

    // element row k-1 (node rows k-1 .. k): Gauss values, f', weights back in y
    float sl[4], sh[4], tl[4], th[4];
#pragma unroll
    for (int s = 0; s < 4; ++s) {
      const float qll = fmaf(kGHi, am1[s], kGLo * am[s]);
      const float qlh = fmaf(kGLo, am1[s], kGHi * am[s]);
      const float qhl = fmaf(kGHi, ap1[s], kGLo * ap[s]);
      const float qhh = fmaf(kGLo, ap1[s], kGHi * ap[s]);
      const float fll = cubic(qll, a.p0, a.p1, a.p2, a.p3);
      const float flh = cubic(qlh, a.p0, a.p1, a.p2, a.p3);
      const float fhl = cubic(qhl, a.p0, a.p1, a.p2, a.p3);
      const float fhh = cubic(qhh, a.p0, a.p1, a.p2, a.p3);
      sl[s] = fmaf(kGHi, fll, fmaf(kGLo, flh, tl1[s]));  // + element row k-2's top share
      sh[s] = fmaf(kGHi, fhl, fmaf(kGLo, fhh, th1[s]));
      tl[s] = fmaf(kGLo, fll, kGHi * flh);
      th[s] = fmaf(kGLo, fhl, kGHi * fhh);
    }
    // weights back in x: node x+v gets segment x+v (left end) and x+v-1 (right end)
    const float sl_l = __shfl_up_sync(kFull, sl[3], 1);
    const float sh_l = __shfl_up_sync(kFull, sh[3], 1);
    float F[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const float pl = (v == 0) ? sl_l : sl[v - 1];
      const float ph = (v == 0) ? sh_l : sh[v - 1];
      F[v] = fmaf(kGHi, sl[v], fmaf(kGLo, sh[v], fmaf(kGLo, pl, kGHi * ph)));
    }

    if constexpr (!kCH) {
      // u(k-1) <- u + F + K1 u   (coefficients carry -dt L / m)
      float o[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        o[v] = c1[v] + F[v] + stencil(a.k1, c2[v], h2[v], c1[v], h1[v], c[v], hs[v]);
      const int row = k - 1;
      if (row >= y0 && row < y0 + kTY && row < ny && lane >= 1 && lane <= 30)
        store_row(a.out + (int64_t)row * nx, x, nx, vec, o);
    } else {
      // mu(k-1) = F + K1 c ; then c(k-2) <- c + K2 mu  (K2 carries -dt M / m)
      float mu[4], mh[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        mu[v] = F[v] + stencil(a.k1, c2[v], h2[v], c1[v], h1[v], c[v], hs[v]);
      const float ml = __shfl_up_sync(kFull, mu[3], 1);
      const float mr = __shfl_down_sync(kFull, mu[0], 1);
      hsum(mu, ml, mr, mh);
      float o[4];
#pragma unroll
      for (int v = 0; v < 4; ++v)
        o[v] = c2[v] + stencil(a.k2, mua[v], mha[v], mub[v], mhb[v], mu[v], mh[v]);
      const int row = k - 2;
      if (row >= y0 && row < y0 + kTY && row < ny && lane >= 1 && lane <= 30)
        store_row(a.out + (int64_t)row * nx, x, nx, vec, o);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        mua[v] = mub[v];
        mha[v] = mhb[v];
        mub[v] = mu[v];
        mhb[v] = mh[v];
      }
    }
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      c2[v] = c1[v];
      h2[v] = h1[v];
      c1[v] = c[v];
      h1[v] = hs[v];
      am1[v] = am[v];
      ap1[v] = ap[v];
      tl1[v] = tl[v];
      th1[v] = th[v];
    }
  }
}

__global__ void k_shift(const float* __restrict__ in, float* __restrict__ out, int64_t n,
                        float add) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    out[i] = in[i] + add;
}

constexpr int kTYAc = 32;
constexpr int kTYCh = 32;

}  // namespace

cudaError_t launch_ac2d(const Explicit2DArgs& a, cudaStream_t s) {
  const dim3 grid((a.nx + kOutCols - 1) / kOutCols, (a.ny + kWarps * kTYAc - 1) / (kWarps * kTYAc));
  k_explicit2d<false, kTYAc><<<grid, kWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_ch2d(const Explicit2DArgs& a, cudaStream_t s) {
  const dim3 grid((a.nx + kOutCols - 1) / kOutCols, (a.ny + kWarps * kTYCh - 1) / (kWarps * kTYCh));
  k_explicit2d<true, kTYCh><<<grid, kWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_shift(const float* in, float* out, int64_t n, float add, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  k_shift<<<(unsigned)blocks, 256, 0, s>>>(in, out, n, add);
  return cudaGetLastError();
}

}  // namespace pf
