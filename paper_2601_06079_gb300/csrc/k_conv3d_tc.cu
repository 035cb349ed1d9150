// 3x3x3 convolution of the learned surrogate on the 5th-generation tensor
// cores: tcgen05.mma (BF16 operands from shared memory, FP32 accumulators in
// tensor memory), input tiles brought in by TMA, warp-specialised pipeline.
//
// Implicit GEMM without an im2col buffer, with the three x-taps folded into
// N.  A block owns a 2x8x14 (z, y, x) output tile.  Per z plane one GEMM
//   D[(y, x'), (dx, co)] = sum over (dz, dy, ci) of X[z+dz, y+dy, x'] W[dz, dy, dx, co, ci]
// runs over the 8 x 16 positions x' of a 16-wide halo row (M = 128) and the
// c_out outputs of all three x-taps (N = 3 c_out, K = 9 c_in); the epilogue
// then adds D[x, dx=0] + D[x+1, dx=1] + D[x+2, dx=2] with two lane shuffles.
// With c_out = 32 every MMA is 128 x 96 x 16 instead of 128 x 32 x 16: a third
// of the instructions for the same work, and fewer shared-memory operand
// bytes per flop.
//
// The input halo (4 x 10 x 16 voxels) is staged by TMA as c_in/8 "chunk
// planes": plane k holds channels 8k..8k+7 of every halo voxel, 16 bytes per
// voxel, voxels in (z, y, x') order.  Eight x'-neighbours are one contiguous
// 128-byte core matrix and a halo row is two of them, so the A operand of
// every (dz, dy) is a shared-memory descriptor at a shifted start address:
// core matrices along M are 128 bytes apart (SBO), along K a plane apart
// (LBO).  The weights of the layer sit in shared memory once per block in the
// same canonical no-swizzle K-major layout ([dz dy][chunk][dx co][8 channels]).
//
// Roles (192 threads): warp 0 issues the TMA loads (3-stage ring) and owns
// the tensor-memory allocation; warp 1 issues the MMAs from one thread and
// commits them to mbarriers; warps 2-5 drain the accumulators
// (tcgen05.ld 32x32b, lane quarter = warp % 4), combine the x-taps, add the
// bias, apply the ReLU and store NDHWC.  Accumulators are double-buffered so
// the epilogue of tile i overlaps the MMAs of tile i+1.  Every wait is
// bounded: on expiry the block records an error code, stops issuing work,
// waits (bounded) for its own copies and MMAs in flight, frees its tensor
// memory and returns.
#include "pf_internal.h"

#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "tc_util.h"

namespace pf {
namespace {

using namespace tc;

constexpr int TZ = 2, TY = 8, TX = 14;                  // output tile
constexpr int HZ = TZ + 2, HY = TY + 2, HX = 16;        // halo tile (16-wide rows)
constexpr uint32_t kPlane = HZ * HY * HX * 16;          // bytes per chunk plane (10240)
#ifndef PF_CONV_SWIZZLE
#define PF_CONV_SWIZZLE 1  // 1: one swizzled voxel-major TMA box per stage; 0: chunk planes
#endif
constexpr int kStages = 3;
constexpr int kThreads = 192;

struct __align__(8) Ctrl {
  uint64_t full[kStages], empty[kStages], accf[2], acce[2], done;
  uint32_t tmem;
  int abort;
};

template <int CIN, int COUT>
struct Cfg {
  static constexpr int kNB = 3 * COUT;  // GEMM N: (dx, c_out)
  static constexpr uint32_t kWBytes = 9u * (CIN / 8) * kNB * 16;
  static constexpr uint32_t kStage = (CIN / 8) * kPlane;
  static constexpr uint32_t kUsed = 2 * TZ * kNB;  // 2 buffers x 2 z planes x N columns
  static constexpr uint32_t kCols = kUsed <= 32 ? 32 : kUsed <= 64 ? 64 : kUsed <= 128 ? 128
                                    : kUsed <= 256 ? 256 : 512;
  // at least 120 KB, so that one block owns an SM and its tensor memory
  static constexpr uint32_t kSmemUse = 1024 + kWBytes + kStages * kStage + sizeof(Ctrl);
  static constexpr uint32_t kSmem = kSmemUse > 120u * 1024 ? kSmemUse : 120u * 1024;
  // kind::f16, FP32 accumulate, BF16 A and B, both K-major, N = 3 COUT, M = 128
  static constexpr uint32_t kIdesc =
      (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kNB >> 3) << 17) | ((128u >> 4) << 24);
  static_assert(kUsed <= 512 && kNB % 16 == 0 && kNB <= 256, "accumulator shape");
};

template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads, 1)
    k_conv3d_tc(const __grid_constant__ CUtensorMap xmap, const __nv_bfloat16* __restrict__ wt,
                const float* __restrict__ bias, int relu, __nv_bfloat16* y16, float* y32, int B,
                int D, int H, int W, int* err, int selftest) {
  using C = Cfg<CIN, COUT>;
  extern __shared__ unsigned char smem_raw[];
  // 128-byte aligned base (TMA destinations and descriptors)
  const uint32_t raw = su32(smem_raw);
  unsigned char* base = smem_raw + ((1024 - (raw & 1023)) & 1023);  // swizzle atoms repeat at 1 KB
  unsigned char* sW = base;
  unsigned char* sIn = base + C::kWBytes;
  Ctrl* ctl = reinterpret_cast<Ctrl*>(sIn + kStages * C::kStage);
  volatile int* abort = &ctl->abort;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tiles_x = (W + TX - 1) / TX, tiles_y = H / TY, tiles_z = D / TZ;
  const int ntiles = B * tiles_z * tiles_y * tiles_x;

  // weights [27][COUT][CIN] -> [9 (dz dy)][CIN/8][3 COUT (dx co)][8]
  for (int i = threadIdx.x; i < 27 * COUT * (CIN / 8); i += kThreads) {
    const int kc = i % (CIN / 8), co = (i / (CIN / 8)) % COUT, tap = i / ((CIN / 8) * COUT);
    const int dzdy = tap / 3, dx = tap % 3;
    *reinterpret_cast<uint4*>(sW + ((dzdy * (CIN / 8) + kc) * C::kNB + dx * COUT + co) * 16) =
        *reinterpret_cast<const uint4*>(wt + (int64_t)i * 8);
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < kStages; ++s) {
      bar_init(&ctl->full[s], 1);
      bar_init(&ctl->empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      bar_init(&ctl->accf[a], 1);
      bar_init(&ctl->acce[a], 128);
    }
    bar_init(&ctl->done, 1);
    ctl->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&ctl->tmem)),
                 "r"(C::kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // weights -> async proxy
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = ctl->tmem;

  if (warp == 0) {
    // ---- TMA producer ----
    // (selftest: issue nothing, so that the MMA thread's bounded wait on the
    // first stage must expire and every role takes the error path)
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntiles && !selftest; t += gridDim.x, ++i) {
        const int s = i % kStages;
        if (i >= kStages && !bar_wait(&ctl->empty[s], ((i / kStages) - 1) & 1, abort, err)) break;
        const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y;
        const int tz = (t / (tiles_x * tiles_y)) % tiles_z, b = t / (tiles_x * tiles_y * tiles_z);
        bar_expect(&ctl->full[s], C::kStage);
        const uint32_t dst = su32(sIn + s * C::kStage);
#if PF_CONV_SWIZZLE
        // one box of whole voxels: [z][y][x'][CIN], rows of CIN * 2 bytes, swizzled
        tma_load5(dst, &xmap, 0, tx * TX - 1, ty * TY - 1, tz * TZ - 1, b, &ctl->full[s]);
#else
#pragma unroll
        for (int k = 0; k < CIN / 8; ++k)
          tma_load5(dst + k * kPlane, &xmap, 8 * k, tx * TX - 1, ty * TY - 1, tz * TZ - 1, b,
                    &ctl->full[s]);
#endif
      }
      // wait (bounded) for the copies still in flight before the block may exit
      const int issued = i;
      for (int s = 0; s < kStages && s < issued; ++s) {
        const int last = s + ((issued - 1 - s) / kStages) * kStages;
        const long long t0 = clock64();
        while (!bar_try(&ctl->full[s], (last / kStages) & 1) && clock64() - t0 < kWaitCycles) {
        }
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer ----
    if (lane == 0) {
      int i = 0;
      for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
        const int s = i % kStages, a = i & 1;
        if (!bar_wait(&ctl->full[s], (i / kStages) & 1, abort, err)) break;
        if (i >= 2 && !bar_wait(&ctl->acce[a], ((i >> 1) - 1) & 1, abort, err)) break;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        // descriptors of the stage / weight bases; every (dz dy, chunk, z) operand
        // is a compile-time byte offset added to the 16-byte address field
#if PF_CONV_SWIZZLE
        // rows = voxels of CIN * 2 bytes, 8-row swizzle atoms 8 CIN * 2 bytes apart
        const uint64_t a_desc =
            sdesc(su32(sIn + s * C::kStage), 16, 8 * CIN * 2, CIN == 32 ? 4ull : 6ull);
#else
        const uint64_t a_desc = sdesc(su32(sIn + s * C::kStage), kPlane, 128);
#endif
        const uint64_t b_desc = sdesc(su32(sW), C::kNB * 16, 128);
        const uint32_t d0 = tmem + a * TZ * C::kNB;
#pragma unroll
        for (int dzdy = 0; dzdy < 9; ++dzdy) {
          const int dz = dzdy / 3, dy = dzdy % 3;
#pragma unroll
          for (int kc = 0; kc < CIN / 16; ++kc) {
            const uint64_t bd =
                b_desc + (uint64_t)(((dzdy * (CIN / 8) + 2 * kc) * C::kNB * 16) >> 4);
#pragma unroll
            for (int z = 0; z < TZ; ++z) {
#if PF_CONV_SWIZZLE
              const uint32_t off = ((z + dz) * HY + dy) * HX * CIN * 2 + kc * 32;
#else
              const uint32_t off = ((z + dz) * HY + dy) * HX * 16 + 2 * kc * kPlane;
#endif
              mma_f16(d0 + z * C::kNB, a_desc + (uint64_t)(off >> 4), bd, C::kIdesc,
                      (dzdy | kc) != 0);
            }
          }
        }
        mma_commit(&ctl->empty[s]);
        mma_commit(&ctl->accf[a]);
      }
      // all MMAs of this block are complete once `done` flips
      mma_commit(&ctl->done);
      const long long t0 = clock64();
      while (!bar_try(&ctl->done, 0) && clock64() - t0 < kWaitCycles) {
      }
    }
  } else {
    // ---- epilogue: warps 2..5, TMEM lane quarter q = warp % 4 ----
    const int q = warp & 3;
    const int row = q * 32 + lane;  // M row = y * 16 + x'
    const int yy = row >> 4, xx = row & 15;
    float bv[COUT];
#pragma unroll
    for (int c = 0; c < COUT; ++c) bv[c] = bias ? bias[c] : 0.0f;
    int i = 0;
    for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++i) {
      const int a = i & 1;
      // warp-uniform outcome: tcgen05.ld below needs the whole warp converged
      const bool ok = bar_wait(&ctl->accf[a], (i >> 1) & 1, abort, err);
      if (!__all_sync(0xffffffffu, ok)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y;
      const int tz = (t / (tiles_x * tiles_y)) % tiles_z, b = t / (tiles_x * tiles_y * tiles_z);
      const int gx = tx * TX + xx;
      const bool store = xx < TX && gx < W;
#pragma unroll
      for (int z = 0; z < TZ; ++z) {
        __syncwarp();  // converged for the .sync.aligned loads after the divergent stores
        const uint32_t col = tmem + ((uint32_t)(q * 32) << 16) + a * TZ * C::kNB + z * C::kNB;
        float v[COUT], w1[COUT], w2[COUT];
        tmem_ld<COUT>(col, v);               // dx = 0, at x' = x
        tmem_ld<COUT>(col + COUT, w1);       // dx = 1, taken from x' = x + 1
        tmem_ld<COUT>(col + 2 * COUT, w2);   // dx = 2, taken from x' = x + 2
#pragma unroll
        for (int c = 0; c < COUT; ++c) {
          v[c] += __shfl_down_sync(0xffffffffu, w1[c], 1) + bv[c];
          v[c] += __shfl_down_sync(0xffffffffu, w2[c], 2);
          if (relu) v[c] = fmaxf(v[c], 0.0f);
        }
        if (store) {
          const int64_t vox = (((int64_t)b * D + tz * TZ + z) * H + ty * TY + yy) * W + gx;
          if (y16) {
            uint4* dst = reinterpret_cast<uint4*>(y16 + vox * COUT);
#pragma unroll
            for (int c = 0; c < COUT / 8; ++c) {
              uint4 o;
              __nv_bfloat162 h0 = __floats2bfloat162_rn(v[8 * c + 0], v[8 * c + 1]);
              __nv_bfloat162 h1 = __floats2bfloat162_rn(v[8 * c + 2], v[8 * c + 3]);
              __nv_bfloat162 h2 = __floats2bfloat162_rn(v[8 * c + 4], v[8 * c + 5]);
              __nv_bfloat162 h3 = __floats2bfloat162_rn(v[8 * c + 6], v[8 * c + 7]);
              o.x = *reinterpret_cast<uint32_t*>(&h0);
              o.y = *reinterpret_cast<uint32_t*>(&h1);
              o.z = *reinterpret_cast<uint32_t*>(&h2);
              o.w = *reinterpret_cast<uint32_t*>(&h3);
              dst[c] = o;
            }
          }
          if (y32) {
            float4* dst = reinterpret_cast<float4*>(y32 + vox * COUT);
#pragma unroll
            for (int c = 0; c < COUT / 4; ++c)
              dst[c] = make_float4(v[4 * c], v[4 * c + 1], v[4 * c + 2], v[4 * c + 3]);
          }
        }
      }
      __syncwarp();
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      bar_arrive(&ctl->acce[a]);
    }
  }

  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  __syncwarp();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(C::kCols));
}

PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// streaming multiprocessors of the current device
cudaError_t sm_count(int& n) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return e == cudaSuccess && n <= 0 ? cudaErrorInvalidDevice : e;
}

template <int CIN, int COUT>
cudaError_t tc_launch(const void* x, const void* wt, const float* bias, int relu, void* y16,
                      float* y32, int B, int D, int H, int W, int* err, int selftest,
                      cudaStream_t s) {
  using C = Cfg<CIN, COUT>;
  auto enc = encode_fn();
  if (!enc) return cudaErrorNotSupported;
  // NDHWC BF16 viewed as 5-D (C, W, H, D, B), innermost first; box = one
  // 8-channel chunk of the 4x18x10 halo; out-of-range voxels read as zero.
  CUtensorMap map;
  const cuuint64_t dims[5] = {(cuuint64_t)CIN, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)D,
                              (cuuint64_t)B};
  const cuuint64_t strides[4] = {(cuuint64_t)CIN * 2, (cuuint64_t)W * CIN * 2,
                                 (cuuint64_t)H * W * CIN * 2, (cuuint64_t)D * H * W * CIN * 2};
#if PF_CONV_SWIZZLE
  const cuuint32_t box[5] = {(cuuint32_t)CIN, HX, HY, HZ, 1};
  const CUtensorMapSwizzle swz = CIN == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B;
#else
  const cuuint32_t box[5] = {8, HX, HY, HZ, 1};
  const CUtensorMapSwizzle swz = CU_TENSOR_MAP_SWIZZLE_NONE;
#endif
  const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  if (enc(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, const_cast<void*>(x), dims, strides, box,
          estr, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
          CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return cudaErrorInvalidValue;
  static std::atomic<unsigned long long> raised{0};
  cudaError_t e = raise_smem_limit(k_conv3d_tc<CIN, COUT>, C::kSmem, raised);
  int sms = 0;
  if (e == cudaSuccess) e = sm_count(sms);
  if (e != cudaSuccess) return e;
  const int ntiles = B * (D / TZ) * (H / TY) * ((W + TX - 1) / TX);
  const int grid = ntiles < sms ? ntiles : sms;
  k_conv3d_tc<CIN, COUT><<<grid, kThreads, C::kSmem, s>>>(
      map, (const __nv_bfloat16*)wt, bias, relu, (__nv_bfloat16*)y16, y32, B, D, H, W, err,
      selftest);
  return cudaGetLastError();
}

}  // namespace

bool conv3d_tc_shape_ok(int B, int D, int H, int W) {
  return B >= 1 && D >= TZ && H >= TY && W >= 1 && D % TZ == 0 && H % TY == 0;
}

cudaError_t launch_conv3d_tc(int cin, int cout, const void* x, const void* wt, const float* bias,
                             int relu, void* y16, float* y32, int B, int D, int H, int W,
                             int* err, cudaStream_t s, int selftest) {
  if (!conv3d_tc_shape_ok(B, D, H, W) || !err || (uintptr_t)x % 16) return cudaErrorInvalidValue;
  if (cin == 16 && cout == 32)
    return tc_launch<16, 32>(x, wt, bias, relu, y16, y32, B, D, H, W, err, selftest, s);
  if (cin == 32 && cout == 32)
    return tc_launch<32, 32>(x, wt, bias, relu, y16, y32, B, D, H, W, err, selftest, s);
  if (cin == 32 && cout == 16)
    return tc_launch<32, 16>(x, wt, bias, relu, y16, y32, B, D, H, W, err, selftest, s);
  return cudaErrorInvalidValue;
}

}  // namespace pf
