// Vector kernels of the Newton-GMRES solver (JAX-PF Eq. 13-14).  The Krylov
// basis is FP32; every inner product and norm is accumulated in FP64: each
// thread forms FP32 partial sums over 8 consecutive products of its stride
// and adds them into FP64 accumulators, blocks reduce in FP64 through shared
// memory, and a single block sums the per-block partials in a fixed order,
// so results are deterministic.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;      // products per FP32 partial sum

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide FP64 sum; the result is valid in thread 0.
__device__ double block_sum(double v, double* scratch) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = v;
  __syncthreads();
  v = (threadIdx.x < kThreads / 32) ? scratch[threadIdx.x] : 0.0;
  if (w == 0) v = warp_sum(v);
  return v;
}

// partials[b * k + j] = sum over block b's indices of V_j . w   (j < k <= kMaxBasis),
// V_j = V + j * ldv; w is read once for all k products.  If w == nullptr the
// squared norm of V_0 is taken (k must be 1).
__global__ void __launch_bounds__(kThreads) k_dots(const float* __restrict__ V, int64_t ldv,
                                                   int k, const float* __restrict__ w, int64_t n,
                                                   double* __restrict__ partials) {
  __shared__ double scratch[kThreads / 32];
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  double acc[kMaxBasis];
#pragma unroll
  for (int j = 0; j < kMaxBasis; ++j) acc[j] = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks;
       c += (int64_t)gridDim.x * kThreads) {
    const int64_t i0 = c * kChunk;
    float u[kChunk];
#pragma unroll
    for (int t = 0; t < kChunk; ++t) u[t] = (i0 + t < n) ? (w ? w[i0 + t] : V[i0 + t]) : 0.0f;
#pragma unroll
    for (int j = 0; j < kMaxBasis; ++j) {
      if (j < k) {
        const float* v = V + j * ldv + i0;
        float s = 0.0f;
#pragma unroll
        for (int t = 0; t < kChunk; ++t)
          if (i0 + t < n) s = fmaf(v[t], u[t], s);
        acc[j] += (double)s;
      }
    }
  }
#pragma unroll
  for (int j = 0; j < kMaxBasis; ++j) {
    if (j < k) {
      const double r = block_sum(acc[j], scratch);
      if (threadIdx.x == 0) partials[blockIdx.x * k + j] = r;
    }
  }
}

// out[j] = sum_b partials[b * k + j], fixed order
__global__ void k_sum_partials_cols(const double* __restrict__ partials, int nblocks, int k,
                                    double* __restrict__ out) {
  __shared__ double scratch[kThreads / 32];
  for (int j = 0; j < k; ++j) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += kThreads) acc += partials[b * k + j];
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) out[j] = acc;
  }
}

// w <- w - sum_j coef[j] V_j (coef: device FP64);  optionally partials of |w|^2
__global__ void __launch_bounds__(kThreads) k_update(const float* __restrict__ V, int64_t ldv,
                                                     int k, const double* __restrict__ coef,
                                                     float* __restrict__ w, int64_t n,
                                                     double* __restrict__ norm_partials) {
  __shared__ double scratch[kThreads / 32];
  __shared__ float cf[kMaxBasis];
  for (int j = threadIdx.x; j < k; j += kThreads) cf[j] = (float)coef[j];
  __syncthreads();
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  double acc = 0.0;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks;
       c += (int64_t)gridDim.x * kThreads) {
    const int64_t i0 = c * kChunk;
    float s = 0.0f;
#pragma unroll
    for (int t = 0; t < kChunk; ++t) {
      const int64_t i = i0 + t;
      if (i < n) {
        float x = w[i];
        for (int j = 0; j < k; ++j) x = fmaf(-cf[j], V[j * ldv + i], x);
        w[i] = x;
        s = fmaf(x, x, s);
      }
    }
    acc += (double)s;
  }
  if (norm_partials) {
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) norm_partials[blockIdx.x] = acc;
  }
}

// y <- a * x + b * y  (host scalars)
__global__ void k_axpby(float a, const float* __restrict__ x, float b, float* __restrict__ y,
                        int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = fmaf(a, x[i], b * y[i]);
}

// x <- x + sum_j y_j V_j
__global__ void k_lincomb(const float* __restrict__ V, int64_t ldv, int k, LinComb y,
                          float* __restrict__ x, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = x[i];
    for (int j = 0; j < k; ++j) s = fmaf(y.c[j], V[j * ldv + i], s);
    x[i] = s;
  }
}

// lumped-mass boundary factor of a node: 1/2 per axis on which it is an end
// node (nz = 1 is a 2-D mesh); node < 2^31 (the mesh limit)
__device__ __forceinline__ float mass_factor(int node, int nx, int ny, int nz) {
  const int x = node % nx, y = (node / nx) % ny, z = node / (nx * ny);
  float m = 1.0f;
  if (x == 0 || x == nx - 1) m *= 0.5f;
  if (y == 0 || y == ny - 1) m *= 0.5f;
  if (nz > 1 && (z == 0 || z == nz - 1)) m *= 0.5f;
  return m;
}

// partials of sum_i (m_i g_i)^2 over all fields: m_i = cell * boundary
// factor.  Products in FP32 (GB300's FP64 rate is a small fraction of its
// FP32 rate), runs of 16 squares in FP32, the runs and the block sum in FP64.
__global__ void __launch_bounds__(kThreads) k_mass_norm(const float* __restrict__ g, int nx,
                                                        int ny, int nz, int nf, float cell,
                                                        double* __restrict__ partials) {
  __shared__ double scratch[kThreads / 32];
  const int N = nx * ny * nz;
  double acc = 0.0;
  float run = 0.0f;
  int k = 0;
  for (int node = blockIdx.x * kThreads + threadIdx.x; node < N; node += gridDim.x * kThreads) {
    const float m = cell * mass_factor(node, nx, ny, nz);
    for (int f = 0; f < nf; ++f) {
      const float v = m * g[(int64_t)f * N + node];
      run = fmaf(v, v, run);
      if (++k == 16) {
        acc += (double)run;
        run = 0.0f;
        k = 0;
      }
    }
  }
  acc += (double)run;
  acc = block_sum(acc, scratch);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc;
}

// out = a * m_i^(+1 or -1) * in over nf planes of nx x ny x nz nodes, m the
// lumped mass (cell times 1/2 per boundary axis; nz = 1 is a 2-D mesh);
// inv_cell = 1 / cell, so that the inverse is a multiplication
__global__ void k_mass_mul(const float* __restrict__ in, float* __restrict__ out, int nx, int ny,
                           int nz, int nf, float cell, float inv_cell, float a, int inverse) {
  const int N = nx * ny * nz;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N; node += gridDim.x * blockDim.x) {
    const float fac = mass_factor(node, nx, ny, nz);
    const float sc = a * (inverse ? inv_cell / fac : cell * fac);  // fac is a power of 2
    for (int f = 0; f < nf; ++f) out[(int64_t)f * N + node] = sc * in[(int64_t)f * N + node];
  }
}

unsigned elementwise_blocks(int64_t n) {
  const int64_t b = (n + 255) / 256, cap = 8 * (int64_t)device_sm_count();
  return (unsigned)(b < cap ? b : cap);
}

}  // namespace

// 3 blocks per SM, fixed per device, so the reductions' order (and result)
// never changes between calls on one device.
int krylov_partial_blocks() { return 3 * device_sm_count(); }

cudaError_t launch_dots(const float* V, int64_t ldv, int k, const float* w, int64_t n,
                        double* partials, double* out, cudaStream_t s) {
  k_dots<<<krylov_partial_blocks(), kThreads, 0, s>>>(V, ldv, k, w, n, partials);
  k_sum_partials_cols<<<1, kThreads, 0, s>>>(partials, krylov_partial_blocks(), k, out);
  return cudaGetLastError();
}

cudaError_t launch_update(const float* V, int64_t ldv, int k, const double* coef, float* w,
                          int64_t n, double* partials, double* norm_out, cudaStream_t s) {
  k_update<<<krylov_partial_blocks(), kThreads, 0, s>>>(V, ldv, k, coef, w, n, norm_out ? partials : nullptr);
  if (norm_out) k_sum_partials_cols<<<1, kThreads, 0, s>>>(partials, krylov_partial_blocks(), 1, norm_out);
  return cudaGetLastError();
}

cudaError_t launch_axpby(float a, const float* x, float b, float* y, int64_t n, cudaStream_t s) {
  k_axpby<<<elementwise_blocks(n), 256, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const float* V, int64_t ldv, int k, const LinComb& y, float* x,
                           int64_t n, cudaStream_t s) {
  k_lincomb<<<elementwise_blocks(n), 256, 0, s>>>(V, ldv, k, y, x, n);
  return cudaGetLastError();
}

cudaError_t launch_mass_mul(const float* in, float* out, int nx, int ny, int nz, int nf,
                            double cell, float a, int inverse, cudaStream_t s) {
  k_mass_mul<<<elementwise_blocks((int64_t)nx * ny * nz), 256, 0, s>>>(
      in, out, nx, ny, nz, nf, (float)cell, (float)(1.0 / cell), a, inverse);
  return cudaGetLastError();
}

cudaError_t launch_mass_norm(const float* g, int nx, int ny, int nz, int nf, double cell,
                             double* partials, double* out, cudaStream_t s) {
  k_mass_norm<<<krylov_partial_blocks(), kThreads, 0, s>>>(g, nx, ny, nz, nf, (float)cell, partials);
  k_sum_partials_cols<<<1, kThreads, 0, s>>>(partials, krylov_partial_blocks(), 1, out);
  return cudaGetLastError();
}

}  // namespace pf
