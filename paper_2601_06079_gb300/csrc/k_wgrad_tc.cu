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
// A block owns tiles of 8 y-rows x 8 x-voxels of one (b, z) plane (H and W are
// multiples of 8); K chunk kb of a tile is its y-row kb.  Eight staging warps
// load 8-voxel x 8-channel blocks (16-byte loads; each thread owns one such
// block of every tile and loads the next tile's while it transposes and stores
// the current one), transpose them in registers and write the
// 128-byte-swizzled K-major layout: every operand row
// holds the tile's 64 voxels in 128 bytes, its 16-byte chunk kb at position
// kb XOR (row mod 8), in atoms of 8 rows (1 KB).  Lanes that store together
// hold different chunks of rows with the same row mod 8, so the swizzle puts
// their 16 bytes in different bank groups (the unswizzled layout put all of
// them in the same one: 8-way conflicts on every store).  The output gradient is loaded once per source row
// (z', y') of the tile's 3 x 10 neighbourhood and stored into every (dy, kb)
// slot it feeds, up to three, rather than once per slot.  Two stages alternate: while the
// staging warps fill one, one thread of warp 8 issues the 4 (K = 16) MMAs per
// group on the other and commits them to the stage's barrier; the K = 16
// steps advance the descriptors' start by 32 bytes within the rows.  Every tile of
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
  static constexpr uint32_t kABytes = 128 * 128;            // one group's A: 128 rows x 128 bytes
  static constexpr uint32_t kBBytes = kN * 128;
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

// byte offset of 16-byte chunk kb (voxels 8 kb .. 8 kb + 7) of operand row r in
// the 128-byte-swizzled K-major layout
__device__ __forceinline__ uint32_t sw128(int r, int kb) {
  return (uint32_t)((r >> 3) * 1024 + (r & 7) * 128 + ((kb ^ (r & 7)) << 4));
}

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
  const int tiles_x = W / 8, tiles_y = H / 8;
  const int64_t ntiles = (int64_t)B * D * tiles_y * tiles_x;

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
    // Thread it owns one block per tile: a source row (dz, yr, c_out chunk) of
    // the output gradient (it < kAItems) or a shifted input row (dx, c_in
    // chunk, kb); source rows vary fastest across lanes, so that lanes storing
    // together differ in kb.
    constexpr int kAItems = 3 * 10 * (COUT / 8);
    constexpr int kBItems = 3 * (CIN / 8) * kKB;
    static_assert(kAItems + kBItems <= kStageWarps * 32, "one block per staging thread");
    const int it = threadIdx.x;
    const bool isA = it < kAItems, active = it < kAItems + kBItems;
    const int yr = it % 10, ca = (it / 10) % (COUT / 8), dz = it / (10 * (COUT / 8));
    const int jb = it - kAItems;
    const int kbb = jb % kKB, cb = (jb / kKB) % (CIN / 8), dxb = jb / (kKB * (CIN / 8));
    const uint4 zero = make_uint4(0, 0, 0, 0);
    // the 8 loads of this thread's block of tile t
    auto load = [&](int64_t t, uint4 (&v)[8]) {
      const int x0 = (int)(t % tiles_x) * 8;
      int64_t r = t / tiles_x;
      const int y0 = (int)(r % tiles_y) * 8;
      r /= tiles_y;
      const int zz = (int)(r % D);
      const int64_t b = r / D;
      if (isA) {
        const int z2 = zz - dz + 1, y2 = y0 - 1 + yr;
        if (z2 >= 0 && z2 < D && y2 >= 0 && y2 < H) {
          const __nv_bfloat16* src = dy + (((b * D + z2) * H + y2) * W + x0) * COUT + 8 * ca;
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = __ldg(reinterpret_cast<const uint4*>(src + k * COUT));
        } else {
#pragma unroll
          for (int k = 0; k < 8; ++k) v[k] = zero;
        }
      } else {
        const int64_t row = (b * D + zz) * H + y0 + kbb;  // (b, z, y) row of the 8 voxels
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int x2 = x0 + k + dxb - 1;
          v[k] = (x2 >= 0 && x2 < W)
                     ? __ldg(reinterpret_cast<const uint4*>(x + (row * W + x2) * CIN + 8 * cb))
                     : zero;
        }
      }
    };
    uint4 nxt[8];
    if (active && blockIdx.x < ntiles) load(blockIdx.x, nxt);
    int i = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int s = i % kStages;
      uint4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = nxt[k];
      if (active && t + gridDim.x < ntiles) load(t + gridDim.x, nxt);  // in flight meanwhile
      if (i >= kStages && !bar_wait(&ctl->empty[s], ((i / kStages) - 1) & 1, abort, err)) break;
      unsigned char* stage = base + s * C::kStage;
      if (active) {
        uint4 o[8];
        transpose8(v, o);
        if (isA) {
          // it feeds slot (dz, dy) at column kb = yr + dy - 2, for every dy with 0 <= kb < 8
#pragma unroll
          for (int dyy = 0; dyy < 3; ++dyy) {
            const int kb = yr + dyy - 2;
            if (kb < 0 || kb >= kKB) continue;
            const int combo = dz * 3 + dyy, g = combo / C::kSPG, sl = combo % C::kSPG;
            unsigned char* dst = stage + g * C::kABytes;
            const int r0 = sl * COUT + 8 * ca;
#pragma unroll
            for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + sw128(r0 + j, kb)) = o[j];
          }
        } else {
          unsigned char* dst = stage + C::kNG * C::kABytes;
          const int r0 = dxb * CIN + 8 * cb;
#pragma unroll
          for (int j = 0; j < 8; ++j) *reinterpret_cast<uint4*>(dst + sw128(r0 + j, kbb)) = o[j];
        }
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
      // 128-byte swizzle (layout 2), 8-row atoms 1 KB apart (SBO); K = 16 steps
      // are 32-byte advances of the start address inside the rows
      const uint64_t b_desc = sdesc(sa + C::kNG * C::kABytes, 16, 1024, 2ull);
#pragma unroll
      for (int g = 0; g < C::kNG; ++g) {
        const uint64_t a_desc = sdesc(sa + g * C::kABytes, 16, 1024, 2ull);
#pragma unroll
        for (int kk = 0; kk < kTile / 16; ++kk)
          mma_f16(tmem + g * C::kN, a_desc + (uint64_t)((32 * kk) >> 4),
                  b_desc + (uint64_t)((32 * kk) >> 4), C::kIdesc, (i > 0 || kk > 0) ? 1u : 0u);
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
  const int64_t ntiles = (int64_t)B * D * (H / 8) * (W / 8);
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
  return B >= 1 && D >= 1 && H >= 8 && W >= 8 && H % 8 == 0 && W % 8 == 0;
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
