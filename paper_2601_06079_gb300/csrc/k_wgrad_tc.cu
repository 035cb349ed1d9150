// Weight gradient of the surrogate's 3x3x3 convolutions on the 5th-generation
// tensor cores (tcgen05.mma, BF16 operands from shared memory, FP32
// accumulators in tensor memory).
//
// With the reduction variable u = v + (dz-1, dy-1, 0) (v the output voxel),
//   dW[dz dy dx][co][ci] = sum over u of dy[u - (dz-1, dy-1, 0)][co] x[u + (0, 0, dx-1)][ci]
// where u runs over the volume only: outside it x (same z, y) or dy (same x)
// is zero.  That is one GEMM per group of (dz, dy) combinations,
//   D_g[(s, co)][(dx, ci)] += A_g[(s, co)][u] B[(dx, ci)][u],
// with M = 128 rows = 128 / c_out combinations s of the group times c_out, and
// N = 3 c_in: the three x-shifts of the input share one B operand, the nine
// (dz, dy) shifts of the output gradient fill the rows of 3 (c_out = 32) or 2
// (c_out = 16) groups, the rows past the ninth combination are zero.
//
// A block owns tiles of 64 consecutive voxels (flattened (b, z, y, x) order;
// W is a multiple of 8, so every 8-voxel run shares z and y).  Eight staging
// warps load the shifted rows (8 voxels x 8 channels, 16-byte loads), transpose
// them in registers and write the canonical no-swizzle K-major layout: core
// matrices of 8 rows x 8 voxels, 8 rows (128 bytes) apart along M/N and the
// operand's rows x 16 bytes apart along K.  Two stages alternate: while the
// staging warps fill one, one thread of warp 8 issues the 4 (K = 16) MMAs per
// group on the other and commits them to the stage's barrier.  Every tile of
// the block accumulates into the same tensor-memory columns (g x 3 c_in + n);
// at the end warps 0..3 (their tensor-memory lane quarters) write the block's
// partial sums, which a second kernel adds over the blocks in a fixed order.
// Every wait is bounded; on expiry the block records an error code, stops,
// waits (bounded) for its own MMAs in flight, frees its tensor memory and
// returns.
#include "pf_internal.h"

#include <cuda_bf16.h>

#include "tc_util.h"

namespace pf {
namespace {

using namespace tc;

constexpr int kTile = 64;        // voxels per tile (K per stage)
constexpr int kKB = kTile / 8;   // 8-voxel core-matrix columns per tile
constexpr int kStageWarps = 8;
constexpr int kThreads = (kStageWarps + 1) * 32;
constexpr int kStages = 2;

template <int CIN, int COUT>
struct WCfg {
  static constexpr int kSPG = 128 / COUT;                  // (dz, dy) combinations per group
  static constexpr int kNG = (9 + kSPG - 1) / kSPG;        // groups
  static constexpr int kN = 3 * CIN;                       // GEMM N: (dx, c_in)
  static constexpr uint32_t kABytes = kKB * 128 * 16;       // one group's A per stage
  static constexpr uint32_t kBBytes = kKB * kN * 16;
  static constexpr uint32_t kStage = kNG * kABytes + kBBytes;
  static constexpr uint32_t kCols = kNG * kN <= 128 ? 128 : kNG * kN <= 256 ? 256 : 512;
  static constexpr uint32_t kSmem = 1024 + kStages * kStage + 256;
  // kind::f16, FP32 accumulate, BF16 A and B, both K-major, N = 3 c_in, M = 128
  static constexpr uint32_t kIdesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) | ((128u >> 4) << 24);
  static_assert(kN % 16 == 0 && kN <= 256 && kNG * kN <= 512, "accumulator shape");
};

struct __align__(8) WCtrl {
  uint64_t full[kStages], empty[kStages], done;
  uint32_t tmem;
  int abort;
};

// 8 x 8 BF16 transpose: in[i] = 8 channels of voxel i; out[j] = 8 voxels of channel j
__device__ __forceinline__ void transpose8(const uint4 (&in)[8], uint4 (&out)[8]) {
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const uint32_t sel = (j & 1) ? 0x7632u : 0x5410u;
    uint32_t w[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t* a = reinterpret_cast<const uint32_t*>(&in[2 * k]);
      const uint32_t* b = reinterpret_cast<const uint32_t*>(&in[2 * k + 1]);
      w[k] = __byte_perm(a[j >> 1], b[j >> 1], sel);
    }
    out[j] = make_uint4(w[0], w[1], w[2], w[3]);
  }
}

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
    k_wgrad_tc(const __nv_bfloat16* __restrict__ x, const __nv_bfloat16* __restrict__ dy,
               float* __restrict__ part, int B, int D, int H, int W, int* err) {
  using C = WCfg<CIN, COUT>;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = su32(smem_raw);
  unsigned char* base = smem_raw + ((1024 - (raw & 1023)) & 1023);
  WCtrl* ctl = reinterpret_cast<WCtrl*>(base + kStages * C::kStage);
  volatile int* abort = &ctl->abort;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t nvox = (int64_t)B * D * H * W;
  const int64_t ntiles = nvox / kTile;

  // zero both stages once: the rows of combinations past the ninth stay zero
  for (uint32_t i = threadIdx.x; i < kStages * C::kStage / 16; i += kThreads)
    reinterpret_cast<uint4*>(base)[i] = make_uint4(0, 0, 0, 0);
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&ctl->full[s], kStageWarps * 32);
      bar_init(&ctl->empty[s], 1);
    }
    bar_init(&ctl->done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kStageWarps) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&ctl->tmem)),
                 "r"(C::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = ctl->tmem;

  if (warp < kStageWarps) {
    // ---- staging: 8 x 8 (voxel, channel) blocks of the shifted operands ----
    const int st = threadIdx.x;
    constexpr int kAItems = 9 * (COUT / 8) * kKB;  // (combination, c_out chunk, column)
    constexpr int kBItems = 3 * (CIN / 8) * kKB;   // (dx, c_in chunk, column)
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int s = i % kStages;
      if (i >= kStages && !bar_wait(&ctl->empty[s], ((i / kStages) - 1) & 1, abort, err)) break;
      unsigned char* stage = base + s * C::kStage;
      const int64_t u0 = t * kTile;
      for (int it = st; it < kAItems + kBItems; it += kStageWarps * 32) {
        uint4 v[8];
        const uint4 zero = make_uint4(0, 0, 0, 0);
        unsigned char* dst;
        uint32_t rows;
        int row0;
        if (it < kAItems) {
          const int kb = it % kKB, c = (it / kKB) % (COUT / 8), combo = it / (kKB * (COUT / 8));
          const int g = combo / C::kSPG, sl = combo % C::kSPG;
          const int64_t u = u0 + kb * 8;
          const int xx = (int)(u % W);
          int64_t r = u / W;
          const int yy = (int)(r % H);
          r /= H;
          const int zz = (int)(r % D);
          const int64_t b = r / D;
          const int z2 = zz - combo / 3 + 1, y2 = yy - combo % 3 + 1;
          if (z2 >= 0 && z2 < D && y2 >= 0 && y2 < H) {
            const __nv_bfloat16* src = dy + (((b * D + z2) * H + y2) * W + xx) * COUT + 8 * c;
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = __ldg(reinterpret_cast<const uint4*>(src + k * COUT));
          } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) v[k] = zero;
          }
          dst = stage + g * C::kABytes + kb * (128 * 16);
          rows = 128;
          row0 = sl * COUT + 8 * c;
        } else {
          const int jb = it - kAItems;
          const int kb = jb % kKB, c = (jb / kKB) % (CIN / 8), dx = jb / (kKB * (CIN / 8));
          const int64_t u = u0 + kb * 8;
          const int xx = (int)(u % W);
          const int64_t row = u / W;  // (b, z, y) row of the 8 voxels
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const int x2 = xx + k + dx - 1;
            v[k] = (x2 >= 0 && x2 < W)
                       ? __ldg(reinterpret_cast<const uint4*>(x + (row * W + x2) * CIN + 8 * c))
                       : zero;
          }
          dst = stage + C::kNG * C::kABytes + kb * (C::kN * 16);
          rows = C::kN;
          row0 = dx * CIN + 8 * c;
        }
        (void)rows;
        uint4 o[8];
        transpose8(v, o);
#pragma unroll
        for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + (row0 + j) * 16) = o[j];
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> MMA
      bar_arrive(&ctl->full[s]);
    }
  } else if (lane == 0) {
    // ---- MMA issuer ----
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int s = i % kStages;
      if (!bar_wait(&ctl->full[s], (i / kStages) & 1, abort, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t sa = su32(base + s * C::kStage);
      const uint64_t b_desc = sdesc(sa + C::kNG * C::kABytes, C::kN * 16, 128);
#pragma unroll
      for (int g = 0; g < C::kNG; ++g) {
        const uint64_t a_desc = sdesc(sa + g * C::kABytes, 128 * 16, 128);
#pragma unroll
        for (int kk = 0; kk < kTile / 16; ++kk)
          mma_f16(tmem + g * C::kN, a_desc + (uint64_t)((2 * kk * 128 * 16) >> 4),
                  b_desc + (uint64_t)((2 * kk * C::kN * 16) >> 4), C::kIdesc,
                  (i > 0 || kk > 0) ? 1u : 0u);
      }
      mma_commit(&ctl->empty[s]);
    }
    mma_commit(&ctl->done);
  }

  // ---- epilogue: warps 0..3 read their lane quarter of every accumulator ----
  if (warp < 4) {
    const bool ok = bar_wait(&ctl->done, 0, abort, err);
    if (__all_sync(0xffffffffu, ok) && blockIdx.x < ntiles) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int m = warp * 32 + lane;
      float* dst = part + ((int64_t)blockIdx.x * C::kNG * 128 + m) * C::kN;
#pragma unroll
      for (int g = 0; g < C::kNG; ++g) {
#pragma unroll
        for (int n0 = 0; n0 < C::kN; n0 += 16) {
          float v[16];
          tmem_ld<16>(tmem + ((uint32_t)(warp * 32) << 16) + g * C::kN + n0, v);
#pragma unroll
          for (int k = 0; k < 16; k += 4)
            *reinterpret_cast<float4*>(dst + (int64_t)g * 128 * C::kN + n0 + k) =
                make_float4(v[k], v[k + 1], v[k + 2], v[k + 3]);
        }
      }
    }
  } else if (warp == kStageWarps && lane == 0) {
    // the MMAs may still be running if the block gave up: wait (bounded)
    const long long t0 = clock64();
    while (!bar_try(&ctl->done, 0) && clock64() - t0 < kWaitCycles) {
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (warp == kStageWarps)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::kCols));
}

// dW[tap][co][ci] = sum over blocks (in order) of part[blk][g][(s, co)][(dx, ci)],
// tap = combination * 3 + dx, combination = g * per-group + s.
template <int CIN, int COUT>
__global__ void k_wgrad_sum(const float* __restrict__ part, int nblk, float* __restrict__ dw) {
  using C = WCfg<CIN, COUT>;
  const int n = 27 * COUT * CIN;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int ci = i % CIN, co = (i / CIN) % COUT, tap = i / (CIN * COUT);
    const int combo = tap / 3, dx = tap % 3;
    const int g = combo / C::kSPG, s = combo % C::kSPG;
    const int64_t off = ((int64_t)g * 128 + s * COUT + co) * C::kN + dx * CIN + ci;
    float acc = 0.0f;
    for (int b = 0; b < nblk; ++b) acc += part[(int64_t)b * C::kNG * 128 * C::kN + off];
    dw[i] = acc;
  }
}

template <int CIN, int COUT>
cudaError_t wgrad_launch(const void* x, const void* dy, float* part, float* dw, int B, int D,
                         int H, int W, int* err, cudaStream_t s) {
  using C = WCfg<CIN, COUT>;
  static std::atomic<unsigned long long> raised{0};
  cudaError_t e = raise_smem_limit(k_wgrad_tc<CIN, COUT>, C::kSmem, raised);
  if (e != cudaSuccess) return e;
  const int64_t ntiles = (int64_t)B * D * H * W / kTile;
  const int grid = (int)(ntiles < wgrad_tc_blocks() ? ntiles : wgrad_tc_blocks());
  k_wgrad_tc<CIN, COUT><<<grid, kThreads, C::kSmem, s>>>(
      (const __nv_bfloat16*)x, (const __nv_bfloat16*)dy, part, B, D, H, W, err);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_wgrad_sum<CIN, COUT><<<(27 * CIN * COUT + 255) / 256, 256, 0, s>>>(part, grid, dw);
  return cudaGetLastError();
}

}  // namespace

int wgrad_tc_blocks() { return device_sm_count(); }

size_t wgrad_tc_part_floats() { return (size_t)wgrad_tc_blocks() * 3 * 128 * 96; }

bool wgrad_tc_shape_ok(int B, int D, int H, int W) {
  return B >= 1 && D >= 1 && H >= 1 && W >= 8 && W % 8 == 0 &&
         ((int64_t)B * D * H * W) % kTile == 0;
}

cudaError_t launch_wgrad_tc(int cin, int cout, const void* x, const void* dy, float* part,
                            float* dw, int B, int D, int H, int W, int* err, cudaStream_t s) {
  if (!wgrad_tc_shape_ok(B, D, H, W) || !err || (uintptr_t)x % 16 || (uintptr_t)dy % 16)
    return cudaErrorInvalidValue;
  if (cin == 16 && cout == 32) return wgrad_launch<16, 32>(x, dy, part, dw, B, D, H, W, err, s);
  if (cin == 32 && cout == 32) return wgrad_launch<32, 32>(x, dy, part, dw, B, D, H, W, err, s);
  if (cin == 32 && cout == 16) return wgrad_launch<32, 16>(x, dy, part, dw, B, D, H, W, err, s);
  return cudaErrorInvalidValue;
}

}  // namespace pf
