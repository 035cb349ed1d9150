// 2-D Cahn-Hilliard with a per-node mobility field: the explicit step and the
// discrete adjoint of that step (JAX-PF Eq. 9-12; sensitivities in the sense
// of Supp. 2, taken through the discrete explicit map).
//
// Forward map (lumped mass m, shifted state d = c - s):
//   mu = m^-1 (F(c) + kappa K c),  c' = c - dt m^-1 K_M mu,
//   (K_M u)_i = sum_e sum_q w|J| M_q grad u_q . grad N_i,  M_q = M sum_a N_a(q) m_a.
// Reverse step for y = m^-1 lambda (lambda = dLoss/dc'):
//   w = m^-1 K_M y,  y_prev = y - dt m^-1 (F'(c) + kappa K) w,
//   dLoss/dM     += -dt / M  sum_i m_i w_i mu_i
//   dLoss/dkappa += -dt sum_i m_i w_i (m^-1 K c)_i
//   dLoss/dW     += -dt / W sum_i m_i w_i (m^-1 F(c))_i
//   dLoss/dm_a   += -dt M sum_e sum_q w|J| N_a(q) grad mu_q . grad y_q
// (F', K, K_M symmetric).  Every operator is evaluated on a block tile staged
// in shared memory with mirror images beyond the mesh, which reproduces the
// zero-flux operators divided by the lumped mass; sums that need the real
// (unmirrored) value at a boundary node take the mirrored value times the
// node's mass fraction.  Reductions are FP64, per block and then in a fixed
// order; per-node gradients accumulate in FP64 in place.  No atomics.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int TX = 32, TY = 16;       // output tile
constexpr int kThreads = 256;
constexpr int S2X = TX + 4, S2Y = TY + 4;  // nodes with a 2-node halo
constexpr int S1X = TX + 2, S1Y = TY + 2;  // nodes with a 1-node halo
constexpr int EX = TX + 3, EY = TY + 3;    // elements touching the 1-halo nodes

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

// Gauss values of a bilinear field from corners c[ay*2+ax]; q = qy*2+qx
__device__ __forceinline__ void qvals(const float c[4], float v[4]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float xi = gpt(q & 1), eta = gpt(q >> 1);
    const float b = fmaf(xi, c[1] - c[0], c[0]), t = fmaf(xi, c[3] - c[2], c[2]);
    v[q] = fmaf(eta, t - b, b);
  }
}

// 1/4 sum_q v_q N_a(q)  (Gauss weight |cell|/4 over the interior mass |cell|)
__device__ __forceinline__ void qproject(const float v[4], float out[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    float s = 0.0f;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const float xi = gpt(q & 1), eta = gpt(q >> 1);
      const float na = ((a & 1) ? xi : 1.0f - xi) * ((a >> 1) ? eta : 1.0f - eta);
      s = fmaf(v[q], na, s);
    }
    out[a] = 0.25f * s;
  }
}

// gradient of a bilinear field at Gauss point q
__device__ __forceinline__ void qgrad(const float c[4], int q, float ihx, float ihy, float& gx,
                                      float& gy) {
  const float xi = gpt(q & 1), eta = gpt(q >> 1);
  gx = ((c[1] - c[0]) * (1.0f - eta) + (c[3] - c[2]) * eta) * ihx;
  gy = ((c[2] - c[0]) * (1.0f - xi) + (c[3] - c[1]) * xi) * ihy;
}

// 1/4 sum_q Mq grad u_q . grad N_a(q)   (mobility-weighted stiffness, scaled)
__device__ __forceinline__ void mob_stiff(const float u[4], const float mq[4], float ihx,
                                          float ihy, float out[4]) {
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] = 0.0f;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const float xi = gpt(q & 1), eta = gpt(q >> 1);
    float gx, gy;
    qgrad(u, q, ihx, ihy, gx, gy);
    gx *= mq[q];
    gy *= mq[q];
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const float dnx = ((a & 1) ? ihx : -ihx) * ((a >> 1) ? eta : 1.0f - eta);
      const float dny = ((a >> 1) ? ihy : -ihy) * ((a & 1) ? xi : 1.0f - xi);
      out[a] = fmaf(gx, dnx, fmaf(gy, dny, out[a]));
    }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) out[a] *= 0.25f;
}

struct Tile {
  float c[S2Y][S2X];   // shifted state d, 2-halo
  float m[S2Y][S2X];   // mobility multiplier, 2-halo
  float y[S2Y][S2X];   // adjoint (reverse step only), 2-halo
  float mu[S1Y][S1X];  // chemical potential, 1-halo
  float w[S1Y][S1X];   // m^-1 K_M y, 1-halo
  float F[S1Y][S1X];   // m^-1 F(c)
  float Kc[S1Y][S1X];  // m^-1 K c (without kappa)
  float E[4][EY][EX];  // per-element corner contributions
  float G[4][EY][EX];  // mobility-gradient corner contributions
};

__device__ __forceinline__ void corners(const float (*a)[S2X], int y, int x, float c[4]) {
  c[0] = a[y][x];
  c[1] = a[y][x + 1];
  c[2] = a[y + 1][x];
  c[3] = a[y + 1][x + 1];
}

__device__ __forceinline__ float gather4(const float (*E)[EY][EX], int y, int x) {
  // node at 2-halo coordinates (y, x): element with corner a has lower-left (y - ay, x - ax)
  return E[0][y][x] + E[1][y][x - 1] + E[2][y - 1][x] + E[3][y - 1][x - 1];
}

__device__ __forceinline__ float stencil9(const float* p, int ld, const Stencil2D& k) {
  return k.c0 * p[0] + k.cx * (p[-1] + p[1]) + k.cy * (p[-ld] + p[ld]) +
         k.cd * (p[-ld - 1] + p[-ld + 1] + p[ld - 1] + p[ld + 1]);
}

// Stage arrays, then F and mu on the 1-halo nodes (shared by both kernels).
__device__ void stage_and_mu(Tile& T, const ChMobArgs& a, const float* yin, int x0, int y0) {
  for (int i = threadIdx.x; i < S2X * S2Y; i += kThreads) {
    const int lx = i % S2X, ly = i / S2X;
    const int64_t g = (int64_t)mirror(y0 - 2 + ly, a.ny) * a.nx + mirror(x0 - 2 + lx, a.nx);
    T.c[ly][lx] = a.d[g];
    T.m[ly][lx] = a.mfield[g];
    if (yin) T.y[ly][lx] = yin[g];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < EX * EY; i += kThreads) {
    const int ex = i % EX, ey = i / EX;
    float c[4], q[4], f[4], o[4];
    corners(T.c, ey, ex, c);
    qvals(c, q);
#pragma unroll
    for (int k = 0; k < 4; ++k) f[k] = fmaf(fmaf(fmaf(a.p3, q[k], a.p2), q[k], a.p1), q[k], a.p0);
    qproject(f, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.E[k][ey][ex] = o[k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < S1X * S1Y; i += kThreads) {
    const int x = 1 + i % S1X, y = 1 + i / S1X;  // 2-halo coordinates
    const float F = gather4(T.E, y, x);
    const float Kc = stencil9(&T.c[y][x], S2X, a.k);
    T.F[y - 1][x - 1] = F;
    T.Kc[y - 1][x - 1] = Kc;
    T.mu[y - 1][x - 1] = fmaf(a.kappa, Kc, F);
  }
  __syncthreads();
}

__device__ __forceinline__ void mob_at(const Tile& T, int ey, int ex, float M, float mq[4]) {
  float mc[4];
  corners(T.m, ey, ex, mc);
  qvals(mc, mq);
#pragma unroll
  for (int k = 0; k < 4; ++k) mq[k] *= M;
}

__global__ void __launch_bounds__(kThreads) k_ch_mob_step(const ChMobArgs a, float* out) {
  __shared__ Tile T;
  const int x0 = blockIdx.x * TX, y0 = block_row() * TY;
  if (y0 >= a.ny) return;
  stage_and_mu(T, a, nullptr, x0, y0);
  // K_M mu on the elements touching the tile nodes (lower-left 1 .. T+1 in 2-halo coords)
  for (int i = threadIdx.x; i < (TX + 1) * (TY + 1); i += kThreads) {
    const int ex = 1 + i % (TX + 1), ey = 1 + i / (TX + 1);
    float u[4], mq[4], o[4];
    u[0] = T.mu[ey - 1][ex - 1];
    u[1] = T.mu[ey - 1][ex];
    u[2] = T.mu[ey][ex - 1];
    u[3] = T.mu[ey][ex];
    mob_at(T, ey, ex, a.M, mq);
    mob_stiff(u, mq, a.ihx, a.ihy, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.E[k][ey][ex] = o[k];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < TX * TY; i += kThreads) {
    const int x = 2 + i % TX, y = 2 + i / TX;
    const int gx = x0 + x - 2, gy = y0 + y - 2;
    if (gx >= a.nx || gy >= a.ny) continue;
    out[(int64_t)gy * a.nx + gx] = fmaf(-a.dt, gather4(T.E, y, x), T.c[y][x]);
  }
}

__global__ void __launch_bounds__(kThreads) k_ch_adj_step(const ChMobArgs a, const float* yin,
                                                          float* yout, float* grad_hi,
                                                          float* grad_lo, double* acc) {
  __shared__ Tile T;
  __shared__ double red[3][kThreads / 32];
  const int x0 = blockIdx.x * TX, y0 = block_row() * TY;
  if (y0 >= a.ny) return;
  stage_and_mu(T, a, yin, x0, y0);
  // K_M y on elements touching the 1-halo nodes; mobility gradient on those
  // touching the tile nodes (mu is known on the 1-halo nodes only)
  for (int i = threadIdx.x; i < EX * EY; i += kThreads) {
    const int ex = i % EX, ey = i / EX;
    float u[4], mq[4], o[4];
    corners(T.y, ey, ex, u);
    mob_at(T, ey, ex, a.M, mq);
    mob_stiff(u, mq, a.ihx, a.ihy, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.E[k][ey][ex] = o[k];
    if (ex >= 1 && ex <= TX + 1 && ey >= 1 && ey <= TY + 1) {
      float mu[4], g[4];
      mu[0] = T.mu[ey - 1][ex - 1];
      mu[1] = T.mu[ey - 1][ex];
      mu[2] = T.mu[ey][ex - 1];
      mu[3] = T.mu[ey][ex];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        float mx, my, yx, yy;
        qgrad(mu, q, a.ihx, a.ihy, mx, my);
        qgrad(u, q, a.ihx, a.ihy, yx, yy);
        g[q] = fmaf(mx, yx, my * yy);
      }
      qproject(g, o);
#pragma unroll
      for (int k = 0; k < 4; ++k) T.G[k][ey][ex] = o[k];
    }
  }
  __syncthreads();
  // per-node products in FP32 (GB300's FP64 rate is a small fraction of its
  // FP32 rate); each thread's two or three nodes sum in FP32, the block sums
  // in FP64.  The running mobility gradient, summed over all steps, is a
  // compensated FP32 pair per node (Knuth's two-sum: the rounding error of
  // each addition is exact in FP32 and collects in lo).  The lumped mass m_i
  // is cell * frac, with cell applied once per thread.
  float dM = 0.0f;
  const float ngm = a.ngm;  // -dt M cell
  for (int i = threadIdx.x; i < S1X * S1Y; i += kThreads) {
    const int x = 1 + i % S1X, y = 1 + i / S1X;
    const float w = gather4(T.E, y, x);
    T.w[y - 1][x - 1] = w;
    const int gx = x0 + x - 2, gy = y0 + y - 2;
    const bool tile_node = x >= 2 && x < TX + 2 && y >= 2 && y < TY + 2;
    if (tile_node && gx < a.nx && gy < a.ny) {
      const float frac = ((gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f) *
                         ((gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f);
      dM = fmaf(frac * w, T.mu[y - 1][x - 1], dM);
      if (grad_hi) {
        const int64_t gi = (int64_t)gy * a.nx + gx;
        const float v = ngm * frac * gather4(T.G, y, x);
        const float hi = grad_hi[gi], t = hi + v, bp = t - hi;
        grad_lo[gi] += (hi - (t - bp)) + (v - bp);
        grad_hi[gi] = t;
      }
    }
  }
  __syncthreads();
  // (F'(c) + kappa K) w on the tile nodes
  for (int i = threadIdx.x; i < (TX + 1) * (TY + 1); i += kThreads) {
    const int ex = 1 + i % (TX + 1), ey = 1 + i / (TX + 1);
    float c[4], cq[4], u[4], uq[4], h[4], o[4];
    corners(T.c, ey, ex, c);
    qvals(c, cq);
    u[0] = T.w[ey - 1][ex - 1];
    u[1] = T.w[ey - 1][ex];
    u[2] = T.w[ey][ex - 1];
    u[3] = T.w[ey][ex];
    qvals(u, uq);
#pragma unroll
    for (int k = 0; k < 4; ++k) h[k] = fmaf(fmaf(a.s2, cq[k], a.s1), cq[k], a.s0) * uq[k];
    qproject(h, o);
#pragma unroll
    for (int k = 0; k < 4; ++k) T.E[k][ey][ex] = o[k];
  }
  __syncthreads();
  float dK = 0.0f, dW = 0.0f;
  for (int i = threadIdx.x; i < TX * TY; i += kThreads) {
    const int x = 2 + i % TX, y = 2 + i / TX;
    const int gx = x0 + x - 2, gy = y0 + y - 2;
    if (gx >= a.nx || gy >= a.ny) continue;
    const float w = T.w[y - 1][x - 1];
    const float Hw = gather4(T.E, y, x) + a.kappa * stencil9(&T.w[y - 1][x - 1], S1X, a.k);
    yout[(int64_t)gy * a.nx + gx] = fmaf(-a.dt, Hw, T.y[y][x]);
    const float frac = ((gx == 0 || gx == a.nx - 1) ? 0.5f : 1.0f) *
                       ((gy == 0 || gy == a.ny - 1) ? 0.5f : 1.0f);
    const float mw = frac * w;
    dK = fmaf(mw, T.Kc[y - 1][x - 1], dK);
    dW = fmaf(mw, T.F[y - 1][x - 1], dW);
  }
  // block sums (fixed order), accumulated across steps in this block's slot:
  // warp sums in FP32 (a shuffle tree per step in FP64 would cost about 20
  // FP64 operations per thread, and GB300 issues 2 per clock per SM), the
  // warps and the steps in FP64
  float v[3] = {dK, dW, dM};
#pragma unroll
  for (int j = 0; j < 3; ++j) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[j] += __shfl_down_sync(0xffffffffu, v[j], o);
    if ((threadIdx.x & 31) == 0) red[j][threadIdx.x >> 5] = a.cell * (double)v[j];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int b = block_row() * gridDim.x + blockIdx.x;
    double s[3] = {0, 0, 0};
    for (int w = 0; w < kThreads / 32; ++w)
      for (int j = 0; j < 3; ++j) s[j] += red[j][w];
    acc[3 * b + 0] += -(double)a.dt * s[0];
    acc[3 * b + 1] += -(double)a.dt * s[1] / a.W;
    acc[3 * b + 2] += -(double)a.dt * s[2] / a.M;
  }
}

// out = hi + lo in FP64 (the compensated FP32 pair of the mobility gradient)
__global__ void k_grad_to_double(const float* __restrict__ hi, const float* __restrict__ lo,
                                 double* __restrict__ out, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (double)hi[i] + (double)lo[i];
}

// loss = 1/2 sum_i wt_i (c_i - t_i)^2 ; y = wt_i (c_i - t_i) / m_i
// (wt = m for the mass-weighted misfit, 1 for the nodal one)
__global__ void k_loss(const float* __restrict__ d, float shift, const float* __restrict__ target,
                       int nx, int ny, double cell, int nodal, float* __restrict__ y,
                       double* __restrict__ partials) {
  __shared__ double red[kThreads / 32];
  const int64_t n = (int64_t)nx * ny;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * kThreads) {
    const int x = (int)(i % nx), yy = (int)(i / nx);
    const double m = cell * ((x == 0 || x == nx - 1) ? 0.5 : 1.0) *
                     ((yy == 0 || yy == ny - 1) ? 0.5 : 1.0);
    const double r = ((double)shift + (double)d[i]) - (double)target[i];
    const double wt = nodal ? 1.0 : m;
    acc += 0.5 * wt * r * r;
    y[i] = (float)(wt * r / m);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// fixed-order sums: out[j] = sum_b in[b * stride + j] for j < k
__global__ void k_colsum(const double* __restrict__ in, int nb, int stride, int k,
                         double* __restrict__ out) {
  if (threadIdx.x < k) {
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += in[(int64_t)b * stride + threadIdx.x];
    out[threadIdx.x] = s;
  }
}

// dLoss/dc0 = m_i y_i
__global__ void k_mass_scale(const float* __restrict__ y, int nx, int ny, double cell,
                             float* __restrict__ out) {
  const int64_t n = (int64_t)nx * ny;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int x = (int)(i % nx), yy = (int)(i / nx);
    const double m = cell * ((x == 0 || x == nx - 1) ? 0.5 : 1.0) *
                     ((yy == 0 || yy == ny - 1) ? 0.5 : 1.0);
    out[i] = (float)(m * (double)y[i]);
  }
}

__global__ void k_add(const float* __restrict__ in, float* __restrict__ out, int64_t n, float add) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] + add;
}

constexpr int kLossBlocks = 256;

}  // namespace

cudaError_t launch_add(const float* in, float* out, int64_t n, float add, cudaStream_t s) {
  int64_t b = (n + 255) / 256;
  k_add<<<(unsigned)(b < 1216 ? b : 1216), 256, 0, s>>>(in, out, n, add);
  return cudaGetLastError();
}

int ch_mob_blocks(int nx, int ny) { return ((nx + TX - 1) / TX) * ((ny + TY - 1) / TY); }

cudaError_t launch_ch_mob_step(const ChMobArgs& a, float* out, cudaStream_t s) {
  const dim3 grid = row_grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  k_ch_mob_step<<<grid, kThreads, 0, s>>>(a, out);
  return cudaGetLastError();
}

cudaError_t launch_ch_adj_step(const ChMobArgs& a, const float* yin, float* yout,
                               float* grad_hi, float* grad_lo, double* acc, cudaStream_t s) {
  if ((grad_hi == nullptr) != (grad_lo == nullptr)) return cudaErrorInvalidValue;
  const dim3 grid = row_grid((a.nx + TX - 1) / TX, (a.ny + TY - 1) / TY);
  k_ch_adj_step<<<grid, kThreads, 0, s>>>(a, yin, yout, grad_hi, grad_lo, acc);
  return cudaGetLastError();
}

cudaError_t launch_grad_to_double(const float* hi, const float* lo, double* out, int64_t n,
                                  cudaStream_t s) {
  int64_t blocks = (n + kThreads - 1) / kThreads;
  if (blocks > 8 * (int64_t)device_sm_count()) blocks = 8 * (int64_t)device_sm_count();
  k_grad_to_double<<<(unsigned)blocks, kThreads, 0, s>>>(hi, lo, out, n);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* d, float shift, const float* target, int nx, int ny,
                        double cell, int nodal, float* y, double* partials, double* out,
                        cudaStream_t s) {
  k_loss<<<kLossBlocks, kThreads, 0, s>>>(d, shift, target, nx, ny, cell, nodal, y, partials);
  k_colsum<<<1, 32, 0, s>>>(partials, kLossBlocks, 1, 1, out);
  return cudaGetLastError();
}

cudaError_t launch_colsum(const double* in, int nb, int stride, int k, double* out,
                          cudaStream_t s) {
  k_colsum<<<1, 32, 0, s>>>(in, nb, stride, k, out);
  return cudaGetLastError();
}

cudaError_t launch_mass_scale(const float* y, int nx, int ny, double cell, float* out,
                              cudaStream_t s) {
  const int64_t n = (int64_t)nx * ny;
  int64_t b = (n + 255) / 256;
  k_mass_scale<<<(unsigned)(b < 1216 ? b : 1216), 256, 0, s>>>(y, nx, ny, cell, out);
  return cudaGetLastError();
}

}  // namespace pf
