// Element-wise layers of the learned surrogate: layout conversions between the
// solver's planar FP32 fields and NDHWC BF16 activations, 2x2x2 average
// pooling, nearest upsampling with an additive skip, ReLU masks, the
// mean-squared loss, weight conversion and the Adam update, each with the
// backward form the training step needs.
#include <algorithm>

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

// 8 BF16 channels (16 bytes) <-> 8 floats
__device__ __forceinline__ void unpack8(const uint4& u, float* f) {
  const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 t = __bfloat1622float2(h[k]);
    f[2 * k] = t.x;
    f[2 * k + 1] = t.y;
  }
}

__device__ __forceinline__ uint4 pack8(const float* f) {
  uint4 u;
  __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&u);
#pragma unroll
  for (int k = 0; k < 4; ++k) h[k] = __floats2bfloat162_rn(f[2 * k], f[2 * k + 1]);
  return u;
}

// planar [B][nf][V] FP32 -> NDHWC BF16 [B][V][C], one thread per voxel (the
// planar reads coalesce across the warp, the voxel's C channels go out as
// 16-byte stores).  mode 0: channels < nf copied, the rest zero.  mode h = 1, 2
// (nf = 8 (h + 1): the states [U^n; U^{n-1}; ...; U^{n-h}]): channels 0..7 =
// U^n, then for k = 1..h the increment (U^{n-k+1} - U^{n-k}) / sig[b], the
// rest zero.
__global__ void k_planar_to_ndhwc(const float* __restrict__ in, int nf, int C, int B, int64_t V,
                                  int mode, const float* __restrict__ sig,
                                  __nv_bfloat16* __restrict__ out) {
  const int64_t n = (int64_t)B * V;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int64_t v = i % V, b = i / V;
    const float inv = mode ? 1.0f / sig[b] : 1.0f;
    uint4* dst = reinterpret_cast<uint4*>(out + i * C);
    for (int c0 = 0; c0 < C; c0 += 8) {
      float f[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int c = c0 + k;
        float a = c < nf ? in[(b * nf + c) * V + v] : 0.0f;
        if (mode && c >= 8 && c < nf) a = (in[(b * nf + c - 8) * V + v] - a) * inv;
        f[k] = a;
      }
      dst[c0 / 8] = pack8(f);
    }
  }
}

// out planar [B][nf][V] = skip + sig[b] * y (first nf channels of the NDHWC
// FP32 y with C channels), sig null = 1.  base: planar with nb channels per
// sample, or null (then mode must be 0).  The skip is mode 0: base[:nf] (U^n);
// mode 1: 2 U^n - U^{n-1} (linear extrapolation); mode 2: 3 U^n - 3 U^{n-1} +
// U^{n-2} (quadratic extrapolation).  One thread per voxel.
__device__ __forceinline__ float skip_value(const float* __restrict__ base, int64_t s0, int64_t st,
                                            int mode) {
  const float u = base[s0];
  if (mode == 1) return 2.0f * u - base[s0 + st];
  if (mode == 2) return fmaf(3.0f, u - base[s0 + st], base[s0 + 2 * st]);
  return u;
}

__global__ void k_ndhwc_to_planar_add(const float* __restrict__ y, int C, int nf, int B, int64_t V,
                                      const float* __restrict__ base, int nb, int mode,
                                      const float* __restrict__ sig, float* __restrict__ out) {
  const int64_t n = (int64_t)B * V;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int64_t v = i % V, b = i / V;
    const float a = sig ? sig[b] : 1.0f;
    const float* src = y + i * C;
    for (int f = 0; f < nf; f += 4) {
      const float4 t = *reinterpret_cast<const float4*>(src + f);
      const float tv[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        if (f + k >= nf) break;
        const float o = base ? skip_value(base, (b * nb + f + k) * V + v, (int64_t)nf * V, mode)
                             : 0.0f;
        out[(b * nf + f + k) * V + v] = fmaf(a, tv[k], o);
      }
    }
  }
}

// Per-sample output unit: sig[b] = a (mode 0) or a * RMS over the sample of
// U^n - U^{n-1} (modes 1, 2: x holds nxc = nf (mode + 1) channels per sample,
// U^n first), floored at 1e-30.  part holds gridDim.x partial sums per sample
// (fixed-order reduction).
//   second = 1 (mode 2): the second difference U^n - 2 U^{n-1} + U^{n-2} instead
__global__ void k_incr_sumsq(const float* __restrict__ x, int nf, int nxc, int64_t V,
                             int second, double* __restrict__ part) {
  __shared__ double red[kT];
  const int b = blockIdx.y;
  const float* u = x + (int64_t)b * nxc * V;
  // differences and squares in FP32 (16-byte loads, four independent sums per
  // thread), runs of 16 vectors summed in FP32 and the runs in FP64: GB300's
  // FP64 rate is a small fraction of its FP32 rate, so no FP64 arithmetic per
  // element.  nf * V is a multiple of 4 (the volume's sides are multiples of 16).
  const float4* u0 = reinterpret_cast<const float4*>(u);
  const float4* u1 = reinterpret_cast<const float4*>(u + nf * V);
  const float4* u2 = reinterpret_cast<const float4*>(u + 2 * nf * V);
  const int64_t n4 = (int64_t)nf * V / 4;
  double acc = 0.0;
  float4 run = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
  int k = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n4;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float4 a0 = u0[i], a1 = u1[i];
    float4 d = make_float4(a0.x - a1.x, a0.y - a1.y, a0.z - a1.z, a0.w - a1.w);
    if (second) {
      const float4 a2 = u2[i];
      d = make_float4(d.x - (a1.x - a2.x), d.y - (a1.y - a2.y), d.z - (a1.z - a2.z),
                      d.w - (a1.w - a2.w));
    }
    run.x = fmaf(d.x, d.x, run.x);
    run.y = fmaf(d.y, d.y, run.y);
    run.z = fmaf(d.z, d.z, run.z);
    run.w = fmaf(d.w, d.w, run.w);
    if (++k == 16) {
      acc += (double)((run.x + run.y) + (run.z + run.w));
      run = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
      k = 0;
    }
  }
  acc += (double)((run.x + run.y) + (run.z + run.w));
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[b * gridDim.x + blockIdx.x] = red[0];
}

// Sum of p[0 .. n) by one block of kT threads in a fixed order (strided
// per-thread sums, then a shared-memory tree), valid in thread 0.  Serial FP64
// adds by one thread wait out the FP64 latency of every add on GB300.
__device__ double block_sum_fixed(const double* __restrict__ p, int n) {
  __shared__ double red[kT];
  double s = 0.0;
  for (int k = threadIdx.x; k < n; k += kT) s += p[k];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  return red[0];
}

// one block per sample
__global__ void __launch_bounds__(kT) k_incr_scale(const double* __restrict__ part, int nblk,
                                                   double count, float a, int mode,
                                                   float* __restrict__ sig) {
  const int b = blockIdx.x;
  if (!mode) {
    if (threadIdx.x == 0) sig[b] = a;
    return;
  }
  const double ss = block_sum_fixed(part + (int64_t)b * nblk, nblk);
  if (threadIdx.x == 0) sig[b] = fmaxf(a * (float)sqrt(ss / count), 1e-30f);
}

// output unit of the quadratic-extrapolation model: a * RMS of the second
// difference, floored at 1e-3 of the increment unit sig[b] (a trajectory
// with no curvature leaves a small correction rather than a vanishing unit);
// one block per sample
__global__ void __launch_bounds__(kT) k_curv_scale(const double* __restrict__ part, int nblk,
                                                   double count, float a,
                                                   const float* __restrict__ sig,
                                                   float* __restrict__ sigo) {
  const int b = blockIdx.x;
  const double ss = block_sum_fixed(part + (int64_t)b * nblk, nblk);
  if (threadIdx.x == 0) sigo[b] = fmaxf(fmaxf(a * (float)sqrt(ss / count), 1e-3f * sig[b]), 1e-30f);
}

// Voxel index helpers for NDHWC: i = ((b * D + z) * H + y) * W + x
struct Vox {
  int64_t b;
  int z, y, x;
};

__device__ __forceinline__ Vox split(int64_t i, int D, int H, int W) {
  Vox v;
  v.x = (int)(i % W);
  i /= W;
  v.y = (int)(i % H);
  i /= H;
  v.z = (int)(i % D);
  v.b = i / D;
  return v;
}

// Sum (scaled) of the 8 fine voxels under every coarse voxel; one thread per
// (coarse voxel, 8-channel chunk).  (D, H, W) are the fine sizes.
__global__ void k_block_sum(const __nv_bfloat16* __restrict__ in, int B, int D, int H, int W,
                            int C, float scale, __nv_bfloat16* __restrict__ out) {
  const int d = D / 2, h = H / 2, w = W / 2, nc = C / 8;
  const int64_t n = (int64_t)B * d * h * w * nc;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % nc);
    const Vox o = split(i / nc, d, h, w);
    float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t src = (((o.b * D + 2 * o.z + (k >> 2)) * H + 2 * o.y + ((k >> 1) & 1)) * W +
                           2 * o.x + (k & 1)) * C + 8 * c;
      float f[8];
      unpack8(*reinterpret_cast<const uint4*>(in + src), f);
#pragma unroll
      for (int j = 0; j < 8; ++j) s[j] += f[j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) s[j] *= scale;
    reinterpret_cast<uint4*>(out)[i] = pack8(s);
  }
}

// out(fine) = acc(fine) + scale * coarse(parent voxel); one thread per (fine
// voxel, 8-channel chunk).  Serves the nearest upsampling + skip of the
// decoder (scale 1) and the backward of the average pooling (scale 1/8).
// acc and out may be the same buffer (in-place accumulation).
__global__ void k_up_add(const __nv_bfloat16* __restrict__ coarse, const __nv_bfloat16* acc,
                         int B, int D, int H, int W, int C, float scale, __nv_bfloat16* out) {
  const int nc = C / 8;
  const int64_t n = (int64_t)B * D * H * W * nc;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % nc);
    const Vox o = split(i / nc, D, H, W);
    const int64_t src =
        (((o.b * (D / 2) + o.z / 2) * (H / 2) + o.y / 2) * (W / 2) + o.x / 2) * C + 8 * c;
    float a[8], f[8];
    unpack8(*reinterpret_cast<const uint4*>(coarse + src), a);
    unpack8(reinterpret_cast<const uint4*>(acc)[i], f);
#pragma unroll
    for (int j = 0; j < 8; ++j) f[j] = fmaf(scale, a[j], f[j]);
    reinterpret_cast<uint4*>(out)[i] = pack8(f);
  }
}

// g <- g * (y > 0)   (ReLU backward, in place), 8 channels per thread
__global__ void k_relu_mask(__nv_bfloat16* __restrict__ g, const __nv_bfloat16* __restrict__ y,
                            int64_t n8) {
  for (int64_t i = gtid(); i < n8; i += grid_stride()) {
    float gv[8], yv[8];
    unpack8(reinterpret_cast<const uint4*>(g)[i], gv);
    unpack8(reinterpret_cast<const uint4*>(y)[i], yv);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (!(yv[j] > 0.0f)) gv[j] = 0.0f;
    reinterpret_cast<uint4*>(g)[i] = pack8(gv);
  }
}

// Error field of the prediction against the target state y = U^{n+1} (planar,
// nf channels) for inputs x (planar, nxc channels, U^n first), with the skip
// of k_ndhwc_to_planar_add:
//   mode 0: r = sig_b * pred - (y - U^n)                       (state units)
//   mode h: r = pred - (y - skip) / sig_b                      (units of sig_b)
// pred = first nf channels of the NDHWC FP32 network output (C channels);
// r is written planar [B][nf][V].
__global__ void k_err(const float* __restrict__ pred, int C, int nf, int nxc, int B, int64_t V,
                      const float* __restrict__ x, const float* __restrict__ y, int mode,
                      const float* __restrict__ sig, float* __restrict__ r) {
  const int64_t n = (int64_t)B * nf * V;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int64_t v = i % V, c = (i / V) % nf, b = i / (nf * V);
    const int64_t s0 = (b * nxc + c) * V + v;
    const float t = y[i] - skip_value(x, s0, (int64_t)nf * V, mode);
    const float p = pred[(b * V + v) * C + c];
    r[i] = mode ? p - t / sig[b] : fmaf(sig[b], p, -t);
  }
}

// out = in + c * (M^-1 K in) on planes of D x H x W nodes (h = 1): K is the
// assembled Q1 stiffness of the unit-spaced mesh (27-point stencil: centre
// 8/3, face neighbours 0, edge neighbours -1/6, corner neighbours -1/12) and
// M its lumped mass; at the boundary the mirror-extended stencil gives M^-1 K
// exactly.  Written as in + c * w * S(in) with S the mirror stencil and
// w = M / h^3 for the symmetric form (I + c K) used by the loss:
//   sym = 0: out = in + c * S(in)            (= (I + c M^-1 K) in)
//   sym = 1: out = in + c * w * S(in)        (= (I + c K) in, symmetric)
__global__ void k_apply_stiff(const float* __restrict__ in, int64_t planes, int D, int H, int W,
                              float c, int sym, float* __restrict__ out) {
  const int64_t V = (int64_t)D * H * W;
  const int64_t n = planes * V;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int64_t p = i / V;
    const int64_t v = i % V;
    const int x = (int)(v % W), y = (int)((v / W) % H), z = (int)(v / ((int64_t)W * H));
    const float* pl = in + p * V;
    float acc = 0.0f;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      int zz = z + dz;
      zz = zz < 0 ? -zz : (zz >= D ? 2 * D - 2 - zz : zz);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        int yy = y + dy;
        yy = yy < 0 ? -yy : (yy >= H ? 2 * H - 2 - yy : yy);
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
          const int k = (dz != 0) + (dy != 0) + (dx != 0);
          if (k == 1) continue;
          const float wgt = k == 0 ? 8.0f / 3.0f : (k == 2 ? -1.0f / 6.0f : -1.0f / 12.0f);
          int xx = x + dx;
          xx = xx < 0 ? -xx : (xx >= W ? 2 * W - 2 - xx : xx);
          acc = fmaf(wgt, pl[((int64_t)zz * H + yy) * W + xx], acc);
        }
      }
    }
    float w = 1.0f;
    if (sym) {
      if (x == 0 || x == W - 1) w *= 0.5f;
      if (y == 0 || y == H - 1) w *= 0.5f;
      if (z == 0 || z == D - 1) w *= 0.5f;
    }
    out[i] = fmaf(c * w, acc, pl[v]);
  }
}

// Per-block partial sums of q^2 over n values.
__global__ void k_sumsq(const float* __restrict__ q, int64_t n, double* __restrict__ partials) {
  __shared__ double red[kT];
  double acc = 0.0;  // runs of 16 squares in FP32, the runs in FP64 (see k_incr_sumsq)
  float run = 0.0f;
  int k = 0;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    run = fmaf(q[i], q[i], run);
    if (++k == 16) {
      acc += (double)run;
      run = 0.0f;
      k = 0;
    }
  }
  acc += (double)run;
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int o = kT / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = red[0];
}

// dL/dpred (NDHWC BF16, C channels, zero beyond nf) from g = dL/dr / 2 (planar):
// 2 * scale * g * dr/dpred with dr/dpred = sig_b (mode 0) or 1 (mode 1).
__global__ void k_grad_out(const float* __restrict__ g, int C, int nf, int B, int64_t V, int mode,
                           const float* __restrict__ sig, float scale,
                           __nv_bfloat16* __restrict__ grad) {
  const int64_t n = (int64_t)B * V * C;
  for (int64_t i = gtid(); i < n; i += grid_stride()) {
    const int c = (int)(i % C);
    float gv = 0.0f;
    if (c < nf) {
      const int64_t v = (i / C) % V, b = i / (C * V);
      gv = 2.0f * scale * g[(b * nf + c) * V + v] * (mode ? 1.0f : sig[b]);
    }
    grad[i] = __float2bfloat16(gv);
  }
}

__global__ void __launch_bounds__(kT) k_sum_doubles(const double* __restrict__ p, int n,
                                                    double scale, double* out) {
  const double s = block_sum_fixed(p, n);
  if (threadIdx.x == 0) *out = s * scale;
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

// Every layer's conversion in one launch: blockIdx.y is the layer, blocks
// stride over its weights (the per-element work of k_convert_weights)
__global__ void k_convert_weights_all(const ConvertTable t) {
  const int l = blockIdx.y;
  const int ci = t.ci[l], co = t.co[l];
  const int64_t n = (int64_t)27 * ci * co;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int c_in = (int)(i % ci), c_out = (int)((i / ci) % co), tap = (int)(i / (ci * co));
    const __nv_bfloat16 v = __float2bfloat16(t.w[l][i]);
    reinterpret_cast<__nv_bfloat16*>(t.fwd[l])[i] = v;
    if (t.bwd[l])
      reinterpret_cast<__nv_bfloat16*>(t.bwd[l])[((int64_t)(26 - tap) * ci + c_in) * co + c_out] = v;
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

cudaError_t launch_planar_to_ndhwc(const float* in, int nf, int C, int B, int64_t V, int mode,
                                   const float* sig, void* out, cudaStream_t s) {
  if (C % 8 || nf > C || (mode && (nf != 8 * (mode + 1) || !sig))) return cudaErrorInvalidValue;
  k_planar_to_ndhwc<<<blocks_for((int64_t)B * V), kT, 0, s>>>(in, nf, C, B, V, mode, sig,
                                                             (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_ndhwc_to_planar_add(const float* y, int C, int nf, int B, int64_t V,
                                       const float* base, int nb, int mode, const float* sig,
                                       float* out, cudaStream_t s) {
  if (C % 4 || nf > C || (mode && (!base || nb < (mode + 1) * nf))) return cudaErrorInvalidValue;
  k_ndhwc_to_planar_add<<<blocks_for((int64_t)B * V), kT, 0, s>>>(y, C, nf, B, V, base, nb, mode,
                                                                 sig, out);
  return cudaGetLastError();
}

cudaError_t launch_incr_scale(const float* x, int nf, int B, int64_t V, float a, int mode,
                              double* part, int nblk, float* sig, float* sigo, cudaStream_t s) {
  if (mode) {
    k_incr_sumsq<<<dim3(nblk, B), kT, 0, s>>>(x, nf, nf * (mode + 1), V, 0, part);
    if (cudaGetLastError() != cudaSuccess) return cudaErrorLaunchFailure;
  }
  k_incr_scale<<<B, kT, 0, s>>>(part, nblk, (double)nf * V, a, mode, sig);
  if (mode == 2) {  // the partials are reused once the increment unit is formed
    k_incr_sumsq<<<dim3(nblk, B), kT, 0, s>>>(x, nf, 3 * nf, V, 1, part);
    k_curv_scale<<<B, kT, 0, s>>>(part, nblk, (double)nf * V, a, sig, sigo);
  } else {
    cudaMemcpyAsync(sigo, sig, sizeof(float) * B, cudaMemcpyDeviceToDevice, s);
  }
  return cudaGetLastError();
}

cudaError_t launch_pool(const void* in, int B, int D, int H, int W, int C, void* out,
                        cudaStream_t s) {
  k_block_sum<<<blocks_for((int64_t)B * D * H * W * C / 64), kT, 0, s>>>(
      (const __nv_bfloat16*)in, B, D, H, W, C, 0.125f, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_up_add(const void* coarse, const void* skip, int B, int D, int H, int W, int C,
                          void* out, cudaStream_t s) {
  k_up_add<<<blocks_for((int64_t)B * D * H * W * C / 8), kT, 0, s>>>(
      (const __nv_bfloat16*)coarse, (const __nv_bfloat16*)skip, B, D, H, W, C, 1.0f,
      (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_down_sum(const void* g, int B, int D, int H, int W, int C, void* out,
                            cudaStream_t s) {
  k_block_sum<<<blocks_for((int64_t)B * D * H * W * C / 64), kT, 0, s>>>(
      (const __nv_bfloat16*)g, B, D, H, W, C, 1.0f, (__nv_bfloat16*)out);
  return cudaGetLastError();
}

cudaError_t launch_pool_back_add(const void* gc, int B, int D, int H, int W, int C, void* acc,
                                 cudaStream_t s) {
  k_up_add<<<blocks_for((int64_t)B * D * H * W * C / 8), kT, 0, s>>>(
      (const __nv_bfloat16*)gc, (const __nv_bfloat16*)acc, B, D, H, W, C, 0.125f,
      (__nv_bfloat16*)acc);
  return cudaGetLastError();
}

cudaError_t launch_relu_mask(void* g, const void* y, int64_t n, cudaStream_t s) {
  if (n % 8) return cudaErrorInvalidValue;
  k_relu_mask<<<blocks_for(n / 8), kT, 0, s>>>((__nv_bfloat16*)g, (const __nv_bfloat16*)y, n / 8);
  return cudaGetLastError();
}

int mse_blocks() { return 1024; }

// loss = scale * sum q^2 with q = (I + c K) r (c = 0: plain squared error),
// r the error field of k_err; dL/dpred follows from dL/dr = 2 scale (I + c K) q.
cudaError_t launch_mse(const float* pred, int C, int nf, int nxc, int B, int D, int H, int W,
                       const float* x, const float* y, int mode, const float* sig, float c,
                       float scale, float* r, float* q, void* grad, double* partials,
                       double* loss, cudaStream_t s) {
  const int64_t V = (int64_t)D * H * W;
  const int64_t n = (int64_t)B * nf * V;
  k_err<<<blocks_for(n), kT, 0, s>>>(pred, C, nf, nxc, B, V, x, y, mode, sig, r);
  const float* qq = r;
  if (c != 0.0f) {
    k_apply_stiff<<<blocks_for(n), kT, 0, s>>>(r, (int64_t)B * nf, D, H, W, c, 1, q);
    qq = q;
  }
  k_sumsq<<<mse_blocks(), kT, 0, s>>>(qq, n, partials);
  k_sum_doubles<<<1, kT, 0, s>>>(partials, mse_blocks(), (double)scale, loss);
  const float* g = qq;
  if (c != 0.0f) {
    k_apply_stiff<<<blocks_for(n), kT, 0, s>>>(q, (int64_t)B * nf, D, H, W, c, 1, r);
    g = r;
  }
  k_grad_out<<<blocks_for((int64_t)B * V * C), kT, 0, s>>>(g, C, nf, B, V, mode, sig, scale,
                                                          (__nv_bfloat16*)grad);
  return cudaGetLastError();
}

cudaError_t launch_convert_weights(const float* w, int ci, int co, void* fwd, void* bwd,
                                   cudaStream_t s) {
  k_convert_weights<<<blocks_for((int64_t)27 * ci * co), kT, 0, s>>>(
      w, ci, co, (__nv_bfloat16*)fwd, (__nv_bfloat16*)bwd);
  return cudaGetLastError();
}

cudaError_t launch_convert_weights_all(const ConvertTable& t, cudaStream_t s) {
  if (t.n < 1 || t.n > kMaxConvertLayers) return cudaErrorInvalidValue;
  int64_t most = 0;
  for (int l = 0; l < t.n; ++l) most = std::max<int64_t>(most, (int64_t)27 * t.ci[l] * t.co[l]);
  k_convert_weights_all<<<dim3((unsigned)((most + kT - 1) / kT), t.n), kT, 0, s>>>(t);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int64_t n, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s) {
  const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
  k_adam<<<blocks_for(n), kT, 0, s>>>(p, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

}  // namespace pf
