// Element-wise layers of the learned surrogate: layout conversions between the
// solver's planar FP32 fields and NDHWC BF16 activations, 2x2x2 average
// pooling, nearest upsampling with an additive skip, ReLU masks, the
// mean-squared loss, weight conversion and the Adam update, each with the
// backward form the training step needs.
#include "pf_internal.h"

#include <cuda_bf16.h>

namespace pf {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ int64_t grid_stride() { return (int64_t)gridDim.x * blockDim.x; }
__device__ __forceinline__ int64_t gtid() { return (int64_t)blockIdx.x * blockDim.x + threadIdx.x; }

unsigned blocks_for(int64_t n) {
  const int64_t b = (n + kT - 1) / kT;
  return (unsigned)(b < 4096 ? b : 4096);
}

// planar [B][nf][V] FP32 -> NDHWC BF16 [B][V][C] (channels >= nf are zero;
// channels k0.. are multiplied by fs)
__global__ void k_planar_to_ndhwc(const float* __restrict__ in, int nf, int C, int B, int64_t V,
                                  int k0, float fs, __nv_bfloat16* __restrict__ out) {
  const int64_t n = (int64_t)B * V * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    const int64_t v = (i / C) % V, b = i / (C * V);
    const float a = c < nf ? in[(b * nf + c) * V + v] : 0.0f;
    out[i] = __float2bfloat16(c < k0 ? a : a * fs);
  }
}

// out planar [B][nf][V] = base + a * first nf channels of y (NDHWC FP32, C
// channels); base is planar with nb channels per sample (its first nf used)
__global__ void k_ndhwc_to_planar_add(const float* __restrict__ y, int C, int nf, int B, int64_t V,
                                      const float* __restrict__ base, int nb, float a,
                                      float* __restrict__ out) {
  const int64_t n = (int64_t)B * nf * V;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int64_t v = i % V, f = (i / V) % nf, b = i / (nf * V);
    out[i] = fmaf(a, y[(b * V + v) * C + f], base ? base[(b * nb + f) * V + v] : 0.0f);
  }
}

// 2x2x2 average pooling, NDHWC, C channels; (D, H, W) are the fine sizes
__global__ void k_pool(const __nv_bfloat16* __restrict__ in, int B, int D, int H, int W, int C,
                       __nv_bfloat16* __restrict__ out) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const int64_t n = (int64_t)B * d * h * w * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    r /= h;
    const int z = (int)(r % d);
    const int64_t b = r / d;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t src = ((((b * D) + 2 * z + (k >> 2)) * H + 2 * y + ((k >> 1) & 1)) * W + 2 * x +
                           (k & 1)) * C + c;
      s += __bfloat162float(in[src]);
    }
    out[i] = __float2bfloat16(0.125f * s);
  }
}

// nearest 2x upsampling of `coarse` plus `skip` (fine sizes D, H, W)
__global__ void k_up_add(const __nv_bfloat16* __restrict__ coarse,
                         const __nv_bfloat16* __restrict__ skip, int B, int D, int H, int W, int C,
                         __nv_bfloat16* __restrict__ out) {
  const int64_t n = (int64_t)B * D * H * W * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int x = (int)(r % W);
    r /= W;
    const int y = (int)(r % H);
    r /= H;
    const int z = (int)(r % D);
    const int64_t b = r / D;
    const int64_t src = ((((b * (D / 2)) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c;
    out[i] = __float2bfloat16(__bfloat162float(coarse[src]) + __bfloat162float(skip[i]));
  }
}

// Backward of up_add and of pool into one fine gradient, and the coarse one:
//   g_fine  = g_out (skip) [+ g_pool_coarse / 8 broadcast]      (fine sizes)
//   g_coarse = sum over each 2x2x2 block of g_out                 (coarse sizes)
__global__ void k_down_sum(const __nv_bfloat16* __restrict__ g, int B, int D, int H, int W, int C,
                           __nv_bfloat16* __restrict__ out) {
  const int d = D / 2, h = H / 2, w = W / 2;
  const int64_t n = (int64_t)B * d * h * w * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int x = (int)(r % w);
    r /= w;
    const int y = (int)(r % h);
    r /= h;
    const int z = (int)(r % d);
    const int64_t b = r / d;
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t src = ((((b * D) + 2 * z + (k >> 2)) * H + 2 * y + ((k >> 1) & 1)) * W + 2 * x +
                           (k & 1)) * C + c;
      s += __bfloat162float(g[src]);
    }
    out[i] = __float2bfloat16(s);
  }
}

// acc (fine) += pool-backward of g_coarse: every fine voxel gets g_coarse / 8
__global__ void k_pool_back_add(const __nv_bfloat16* __restrict__ gc, int B, int D, int H, int W,
                                int C, __nv_bfloat16* __restrict__ acc) {
  const int64_t n = (int64_t)B * D * H * W * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    int64_t r = i / C;
    const int x = (int)(r % W);
    r /= W;
    const int y = (int)(r % H);
    r /= H;
    const int z = (int)(r % D);
    const int64_t b = r / D;
    const int64_t src = ((((b * (D / 2)) + z / 2) * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c;
    acc[i] = __float2bfloat16(__bfloat162float(acc[i]) + 0.125f * __bfloat162float(gc[src]));
  }
}

// g <- g * (y > 0)   (ReLU backward, in place)
__global__ void k_relu_mask(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ y,
                            int64_t n) {
  for (int64_t i = gtid(); i < n; i += grid_stride())
    if (!(__bfloat162float(y[i]) > 0.0f)) g[i] = __float2bfloat16(0.0f);
}

// Mean-squared loss between a * (first nf channels of pred) (NDHWC FP32, C ch)
// and target = y - x (planar FP32, x with nx channels of which the first nf
// are the state); writes dL/dpred (NDHWC BF16, zero beyond nf) and per-block
// partial sums of the squared error.
__global__ void k_mse(const float* __restrict__ pred, int C, int nf, int nxc, int B, int64_t V,
                      const float* __restrict__ x, const float* __restrict__ y, float a,
                      float scale, __nv_bfloat16* __restrict__ grad,
                      double* __restrict__ partials) {
  __shared__ double red[kT];
  double acc = 0.0;
  const int64_t n = (int64_t)B * V * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    float gval = 0.0f;
    if (c < nf) {
      const int64_t v = (i / C) % V, b = i / (C * V);
      const int64_t p = (b * nf + c) * V + v;
      const float r = fmaf(a, pred[i], -(y[p] - x[(b * nxc + c) * V + v]));
      acc += (double)r * r;
      gval = 2.0f * scale * a * r;
    }
    grad[i] = __float2bfloat16(gval);
  }
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

__global__ void k_sum_doubles(const double* __restrict__ p, int n, double scale, double* out) {
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < n; ++i) s += p[i];
    *out = s * scale;
  }
}

// master FP32 weights [27][co][ci] -> BF16 forward copy and the data-gradient
// copy [27][ci][co] with the taps reversed
__global__ void k_convert_weights(const float* __restrict__ w, int ci, int co,
                                  __nv_bfloat16* __restrict__ fwd, __nv_bfloat16* __restrict__ bwd) {
  const int64_t n = (int64_t)27 * ci * co;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c_in = (int)(i % ci), c_out = (int)((i / ci) % co), tap = (int)(i / (ci * co));
    const __nv_bfloat16 v = __float2bfloat16(w[i]);
    fwd[i] = v;
    if (bwd) bwd[((int64_t)(26 - tap) * ci + c_in) * co + c_out] = v;
  }
}

// Adam (Kingma & Ba 2015) with bias correction; g holds the gradient
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       const float* __restrict__ g, int64_t n, float lr, float b1, float b2,
                       float eps, float c1, float c2) {
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  }
}

}  // namespace

cudaError_t launch_planar_to_ndhwc(const float* in, int nf, int C, int B, int64_t V, int k0,
                                   float fs, void* out, cudaStream_t s) {
  k_planar_to_ndhwc<<<blocks_for((int64_t)B * V * C), kT, 0, s>>>(in, nf, C, B, V, k0, fs,
                                                                  (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_ndhwc_to_planar_add(const float* y, int C, int nf, int B, int64_t V,
                                       const float* base, int nb, float a, float* out,
                                       cudaStream_t s) {
  k_ndhwc_to_planar_add<<<blocks_for((int64_t)B * nf * V), kT, 0, s>>>(y, C, nf, B, V, base, nb,
                                                                      a, out);
  return cudaGetLastError();
}

cudaError_t launch_pool(const void* in, int B, int D, int H, int W, int C, void* out,
                        cudaStream_t s) {
  k_pool<<<blocks_for((int64_t)B * D * H * W * C / 8), kT, 0, s>>>(
      (const __nv_bfloat16*)in, B, D, H, W, C, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_up_add(const void* coarse, const void* skip, int B, int D, int H, int W, int C,
                          void* out, cudaStream_t s) {
  k_up_add<<<blocks_for((int64_t)B * D * H * W * C), kT, 0, s>>>(
      (const __nv_bfloat16*)coarse, (const __nv_bfloat16*)skip, B, D, H, W, C, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_down_sum(const void* g, int B, int D, int H, int W, int C, void* out,
                            cudaStream_t s) {
  k_down_sum<<<blocks_for((int64_t)B * D * H * W * C / 8), kT, 0, s>>>(
      (const __nv_bfloat16*)g, B, D, H, W, C, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_pool_back_add(const void* gc, int B, int D, int H, int W, int C, void* acc,
                                 cudaStream_t s) {
  k_pool_back_add<<<blocks_for((int64_t)B * D * H * W * C), kT, 0, s>>>(
      (const __nv_bfloat16*)gc, B, D, H, W, C, (__nv_bfloat16*)acc);
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(void* g, const void* y, int64_t n, cudaStream_t s) {
  k_relu_mask<<<blocks_for(n), kT, 0, s>>>((__nv_bfloat16*)g, (const __nv_bfloat16*)y, n);
  return cudaGetLastError();
}

int mse_blocks() { return 1024; }

cudaError_t launch_mse(const float* pred, int C, int nf, int nxc, int B, int64_t V,
                       const float* x, const float* y, float a, float scale, void* grad,
                       double* partials, double* loss, cudaStream_t s) {
  k_mse<<<mse_blocks(), kT, 0, s>>>(pred, C, nf, nxc, B, V, x, y, a, scale, (__nv_bfloat16*)grad,
                                    partials);
  k_sum_doubles<<<1, 32, 0, s>>>(partials, mse_blocks(), (double)scale, loss);
  return cudaGetLastError();
}

cudaError_t launch_convert_weights(const float* w, int ci, int co, void* fwd, void* bwd,
                                   cudaStream_t s) {
  k_convert_weights<<<blocks_for((int64_t)27 * ci * co), kT, 0, s>>>(
      w, ci, co, (__nv_bfloat16*)fwd, (__nv_bfloat16*)bwd);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int64_t n, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<blocks_for(n), kT, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace pf
