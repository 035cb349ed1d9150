// FP64 diagnostics: discrete free energy E_h (JAX-PF Eq. 5-6 with the 2x2
// Gauss rule) and the mass integral sum_i m_i u_i with the lumped mass.
// Per-element values are formed in FP32 from the shifted state and summed
// in FP64: warp shuffles, then shared memory, one partial per block, then a
// single-block pass over the partials in a fixed order, so the result does
// not depend on scheduling (no atomics).
#include <math.h>

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

// ---------------------------------------------------------------------------
// Energy / mass without a context or a workspace (pf_energy2d_static).
//
// Some callers cannot allocate device memory: a host that owns all device
// memory through its own allocator and forbids foreign allocations, a process
// that runs under a fixed device-memory budget, or a latency-critical path
// where cudaMalloc / cudaFree would synchronise the whole device.  For them
// the reduction's scratch -- one FP64 (energy, mass) pair per block of the
// first pass -- sits in the static array below instead of a caller-bound
// workspace.  Its size is fixed: kMaxBlocks pairs (16 KiB), which is every
// block the first pass ever launches, so any mesh the kernel accepts fits.
// Every GPU that loads libpf holds this array until the process exits.
// ---------------------------------------------------------------------------
#include <mutex>

namespace pf {
namespace {

static __device__ __align__(256) double g_static_partials[2 * kMaxBlocks];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double* g_static_ptr[kMaxDevices] = {};

// Device address of g_static_partials for the current device, looked up once
// per device (host code only knows the symbol as a host-side stand-in).  The
// cache lives as long as the process; a cudaDeviceReset invalidates it, which
// the header states as a usage rule.
cudaError_t static_partials(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_ptr[dev]) {
    double* p = nullptr;
    e = cudaGetSymbolAddress((void**)&p, g_static_partials);
    if (e != cudaSuccess) return e;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
  return cudaSuccess;
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_energy2d_static(const float* state, int64_t nx, int64_t ny, double hx,
                                        double hy, double W, double kappa, double* out,
                                        void* stream, const char** err) {
  const char* msg = nullptr;
  if (!state || !out) msg = "state and out must be non-null device pointers";
  else if (nx < 2 || ny < 2) msg = "nx and ny must be >= 2";
  else if (nx > INT32_MAX || ny > INT32_MAX || nx * ny > (int64_t)INT32_MAX)
    msg = "mesh too large: nx * ny must be <= 2^31 - 1 nodes";
  else if (!(hx > 0.0) || !(hy > 0.0) || !isfinite(hx) || !isfinite(hy))
    msg = "hx and hy must be finite and > 0";
  else if (!isfinite(W) || !isfinite(kappa)) msg = "W and kappa must be finite";
  if (msg) {
    if (err) *err = msg;
    return PF_ERR_ARG;
  }
  double* partials = nullptr;
  cudaError_t e = pf::static_partials(&partials);
  if (e == cudaSuccess) {
    pf::Energy2DArgs a{};
    a.d = state;
    a.nx = (int)nx;
    a.ny = (int)ny;
    a.hx = hx;
    a.hy = hy;
    a.shift = 0.0f;
    a.q2 = (float)W;
    a.q3 = (float)(-2 * W);
    a.q4 = (float)W;
    a.kappa = (float)kappa;
    e = pf::launch_energy2d(a, partials, out, (cudaStream_t)stream);
  }
  if (e != cudaSuccess) {
    if (err) *err = cudaGetErrorString(e);
    return PF_ERR_CUDA;
  }
  if (err) *err = "";
  return PF_OK;
}

// ---------------------------------------------------------------------------
// Squared distance sum_i (a_i - b_i)^2 (pf_sq_distance).
//
// Each difference d is formed in FP32 and its square split exactly into
// p = fl(d * d) and e = fma(d, d, -p).  A thread keeps a compensated FP32 pair
// (Knuth's two-sum on the running value, rounding errors and e into the low
// word), so no FP64 operation runs per element; the pair enters the FP64 block
// sum once, and the block partials are summed by one block in a fixed order.
// ---------------------------------------------------------------------------
namespace pf {
namespace {

__global__ void __launch_bounds__(kThreads) k_sq_distance(const float* a, const float* b,
                                                          int64_t n, double* partials) {
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  float hi = 0.0f, lo = 0.0f;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < n; i += stride) {
    const float d = a[i] - b[i];
    const float p = __fmul_rn(d, d);  // never contracted into the add below
    const float e = fmaf(d, d, -p);
    const float s = hi + p;
    const float bp = s - hi;
    lo += ((hi - (s - bp)) + (p - bp)) + e;
    hi = s;
  }
  double v = (double)hi + (double)lo, unused = 0.0;
  block_sum2(v, unused);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = v;
    partials[2 * blockIdx.x + 1] = 0.0;
  }
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_sq_distance(const float* a, const float* b, int64_t n,
                                    double* dev_scratch, void* stream, double* out) {
  if (!out || n < 0 || (n > 0 && (!a || !b || !dev_scratch))) return PF_ERR_ARG;
  *out = 0.0;
  if (n == 0) return PF_OK;
  const cudaStream_t s = (cudaStream_t)stream;
  const int64_t want = (n + pf::kThreads - 1) / pf::kThreads;
  const int nb = (int)(want < pf::kMaxBlocks ? want : pf::kMaxBlocks);
  double* result = dev_scratch + 2 * pf::kMaxBlocks;
  pf::k_sq_distance<<<nb, pf::kThreads, 0, s>>>(a, b, n, dev_scratch);
  pf::k_sum_partials<<<1, pf::kThreads, 0, s>>>(dev_scratch, nb, result);
  double host = 0.0;
  if (cudaGetLastError() != cudaSuccess ||
      cudaMemcpyAsync(&host, result, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PF_ERR_CUDA;
  *out = host;
  return PF_OK;
}
