// Measured FP32 FMA throughput of the device (pf_fp32_peak).  The ALU
// rooflines of the explicit step, the JVP and the elastic stiffness are
// stated against this number, taken on the same GPU in the same run, rather
// than against units x clock.  Every thread runs kChains independent chains
// of packed FP32 FMAs (fma.rn.f32x2: two FP32 FMAs per lane per instruction),
// so the FMA pipe, not instruction latency, sets the rate; the grid fills
// every SM at full occupancy.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kThreads = 256;
constexpr int kChains = 8;
constexpr int kIters = 4096;

__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}

__global__ void __launch_bounds__(kThreads) k_fma_peak(float seed, float* sink) {
  unsigned long long acc[kChains], m, c;
  const float s = seed + 1e-7f * (float)threadIdx.x;
  asm("mov.b64 %0, {%1, %1};" : "=l"(m) : "f"(0.999999f));
  asm("mov.b64 %0, {%1, %1};" : "=l"(c) : "f"(1e-7f));
#pragma unroll
  for (int k = 0; k < kChains; ++k) asm("mov.b64 %0, {%1, %2};" : "=l"(acc[k]) : "f"(s + k), "f"(s - k));
  for (int i = 0; i < kIters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) acc[k] = fma2(acc[k], m, c);
  }
  float tot = 0.0f;
#pragma unroll
  for (int k = 0; k < kChains; ++k) {
    float lo, hi;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(acc[k]));
    tot += lo + hi;
  }
  if (tot == 12345.678f) sink[0] = tot;  // keeps the chains live; never true in practice
}

}  // namespace
}  // namespace pf

extern "C" pf_status pf_fp32_peak(void* stream, float* dev_sink, double* tflops) {
  if (!dev_sink || !tflops) return PF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  int per = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, pf::k_fma_peak, pf::kThreads, 0) !=
          cudaSuccess)
    return PF_ERR_CUDA;
  const int grid = 4 * (per < 1 ? 1 : per) * pf::device_sm_count();
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return PF_ERR_CUDA;
  float best = 1e30f;
  cudaError_t e = cudaSuccess;
  for (int r = 0; r < 4 && e == cudaSuccess; ++r) {  // the first launch warms up
    e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
      pf::k_fma_peak<<<grid, pf::kThreads, 0, s>>>(0.5f, dev_sink);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && ms < best) best = ms;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return PF_ERR_CUDA;
  // per thread: kIters x kChains packed FMAs = 2 FMAs = 4 flop each
  const double flop = 4.0 * pf::kIters * pf::kChains * (double)grid * pf::kThreads;
  *tflops = flop / (best * 1e-3) / 1e12;
  return PF_OK;
}
