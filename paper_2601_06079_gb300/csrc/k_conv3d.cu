// Kernels of the learned 3-D surrogate (warm start for the implicit step):
// 3x3x3 convolution (stride 1, zero padding 1) as an implicit GEMM on the
// tensor cores, BF16 operands, FP32 accumulation, plus the layers around it.
//
// Activations are NDHWC BF16 with 16 or 32 channels (the 8 order parameters
// are padded to 16).  A block computes a 2x8x8 output tile for all output
// channels: the input tile with its halo (4x10x10 voxels) and the layer's
// weights sit in shared memory; each of the 4 warps owns 32 output voxels
// (two m16 fragments).  For every tap and 16-channel slice the A fragment is
// gathered straight from the shifted halo tile with ldmatrix (one row address
// per lane), the B fragment comes from the [tap][c_out][c_in] weight block,
// and mma.sync m16n8k16 accumulates in FP32.  Blocks are persistent over the
// output tiles so the weights are staged once per block.
//
// Backward: the data gradient is the same kernel applied to dy with the taps
// flipped and the channel roles swapped; the weight gradient is a GEMM over
// voxels with both operands transposed by ldmatrix.trans, reduced per block
// and then over blocks in a fixed order.
#include "pf_internal.h"

#include <cuda_bf16.h>

namespace pf {
namespace {

constexpr int TZ = 2, TY = 8, TX = 8;                 // output tile
constexpr int HZ = TZ + 2, HY = TY + 2, HX = TX + 2;  // with halo
constexpr int kHalo = HZ * HY * HX;                   // 400 voxels
constexpr int kThreads = 128;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                        unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned& r0, unsigned& r1, unsigned& r2,
                                          unsigned& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

__device__ __forceinline__ void mma_bf16(float* d, unsigned a0, unsigned a1, unsigned a2,
                                         unsigned a3, unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, "
      "{%4, %5, %6, %7}, {%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// voxel (z, y, x) of a block's output tile from the row index m = (z*TY + y)*TX + x
__device__ __forceinline__ int halo_index(int m, int dz, int dy, int dx) {
  const int z = m / (TY * TX), y = (m / TX) % TY, x = m % TX;
  return ((z + dz) * HY + (y + dy)) * HX + (x + dx);
}

// Stage the input tile with its halo (zero outside the volume).  CS = padded
// channel stride in smem (halves).
template <int CIN, int CS>
__device__ void stage_tile(__nv_bfloat16* sIn, const __nv_bfloat16* __restrict__ x, int b, int oz,
                           int oy, int ox, int D, int H, int W) {
  constexpr int kChunks = CIN / 8;  // 16-byte chunks per voxel
  for (int i = threadIdx.x; i < kHalo * kChunks; i += kThreads) {
    const int v = i / kChunks, c = i % kChunks;
    const int hx = v % HX, hy = (v / HX) % HY, hz = v / (HX * HY);
    const int gz = oz + hz - 1, gy = oy + hy - 1, gx = ox + hx - 1;
    uint4 val = make_uint4(0, 0, 0, 0);
    if (gz >= 0 && gz < D && gy >= 0 && gy < H && gx >= 0 && gx < W)
      val = *reinterpret_cast<const uint4*>(
          x + ((((int64_t)b * D + gz) * H + gy) * W + gx) * CIN + c * 8);
    *reinterpret_cast<uint4*>(sIn + v * CS + c * 8) = val;
  }
}

// y = conv(x) (+ bias) (ReLU); weights wt[27][COUT][CIN] BF16.  Output BF16
// NDHWC (y16) and/or FP32 NDHWC (y32).
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv3d(const __nv_bfloat16* __restrict__ x,
                                                     const __nv_bfloat16* __restrict__ wt,
                                                     const float* __restrict__ bias, int relu,
                                                     __nv_bfloat16* y16, float* y32, int B, int D,
                                                     int H, int W) {
  constexpr int CS = CIN + 8;  // padded channel stride (halves): conflict-free ldmatrix rows
  constexpr int NT = COUT / 8;  // n8 fragments
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __nv_bfloat16* sW = reinterpret_cast<__nv_bfloat16*>(smem_raw);  // [27][COUT][CS]
  __nv_bfloat16* sIn = sW + 27 * COUT * CS;                          // [kHalo][CS]

  for (int i = threadIdx.x; i < 27 * COUT * (CIN / 8); i += kThreads) {
    const int row = i / (CIN / 8), c = i % (CIN / 8);
    *reinterpret_cast<uint4*>(sW + row * CS + c * 8) =
        *reinterpret_cast<const uint4*>(wt + (int64_t)row * CIN + c * 8);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tiles_x = W / TX, tiles_y = H / TY, tiles_z = D / TZ;
  const int ntiles = B * tiles_z * tiles_y * tiles_x;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y, tz = (t / (tiles_x * tiles_y)) % tiles_z;
    const int b = t / (tiles_x * tiles_y * tiles_z);
    const int oz = tz * TZ, oy = ty * TY, ox = tx * TX;
    __syncthreads();  // previous tile's readers are done with sIn
    stage_tile<CIN, CS>(sIn, x, b, oz, oy, ox, D, H, W);
    __syncthreads();

    float acc[2][NT][4];
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int nt = 0; nt < NT; ++nt)
#pragma unroll
        for (int k = 0; k < 4; ++k) acc[mt][nt][k] = 0.0f;

    // A rows of this lane: row r of each m16 fragment, k offset 0 or 8
    const int r = ((lane >> 3) & 1) * 8 + (lane & 7);
    const int ka = (lane >> 4) * 8;
    const int m0 = warp * 32 + r, m1 = warp * 32 + 16 + r;
    // B rows (ldmatrix x4 over two n8 fragments): n row, k offset
    const int nb = ((lane >> 4) & 1) * 8 + (lane & 7);
    const int kb = ((lane >> 3) & 1) * 8;

    for (int tap = 0; tap < 27; ++tap) {
      const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
      const __nv_bfloat16* a0p = sIn + halo_index(m0, dz, dy, dx) * CS + ka;
      const __nv_bfloat16* a1p = sIn + halo_index(m1, dz, dy, dx) * CS + ka;
#pragma unroll
      for (int kc = 0; kc < CIN / 16; ++kc) {
        unsigned a[2][4];
        ldsm_x4(smem_u32(a0p + kc * 16), a[0][0], a[0][1], a[0][2], a[0][3]);
        ldsm_x4(smem_u32(a1p + kc * 16), a[1][0], a[1][1], a[1][2], a[1][3]);
#pragma unroll
        for (int np = 0; np < NT / 2; ++np) {
          unsigned b0, b1, b2, b3;
          ldsm_x4(smem_u32(sW + (tap * COUT + np * 16 + nb) * CS + kc * 16 + kb), b0, b1, b2, b3);
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            mma_bf16(acc[mt][2 * np], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b0, b1);
            mma_bf16(acc[mt][2 * np + 1], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b2, b3);
          }
        }
      }
    }
    // epilogue: fragment element (row g or g+8, column 2 tig + {0,1})
    const int g = lane >> 2, tig = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt)
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int m = warp * 32 + mt * 16 + half * 8 + g;
        const int z = m / (TY * TX), yy = (m / TX) % TY, xx = m % TX;
        const int64_t vox = (((int64_t)b * D + oz + z) * H + oy + yy) * W + ox + xx;
#pragma unroll
        for (int nt = 0; nt < NT; ++nt) {
          const int c = nt * 8 + 2 * tig;
          float v0 = acc[mt][nt][2 * half], v1 = acc[mt][nt][2 * half + 1];
          if (bias) {
            v0 += bias[c];
            v1 += bias[c + 1];
          }
          if (relu) {
            v0 = fmaxf(v0, 0.0f);
            v1 = fmaxf(v1, 0.0f);
          }
          if (y16)
            *reinterpret_cast<__nv_bfloat162*>(y16 + vox * COUT + c) = __floats2bfloat162_rn(v0, v1);
          if (y32) *reinterpret_cast<float2*>(y32 + vox * COUT + c) = make_float2(v0, v1);
        }
      }
  }
}

// Weight gradient: part[blk][tap][co][ci] = sum over this block's voxels of
// dy[v][co] * x[v + tap - 1][ci].  Each block owns 3 taps (one (kz, ky) row)
// and strides over voxel tiles; warp w owns output fragments w, w+4, ...
template <int CIN, int COUT>
__global__ void __launch_bounds__(kThreads) k_conv3d_wgrad(const __nv_bfloat16* __restrict__ x,
                                                           const __nv_bfloat16* __restrict__ dy,
                                                           float* __restrict__ part, int B, int D,
                                                           int H, int W) {
  constexpr int CS = CIN + 8, DS = COUT + 8;
  constexpr int MT = COUT / 16, NT = CIN / 8;  // output fragments: MT x NT per tap
  constexpr int FR = 3 * MT * NT;              // fragments per block (3 taps)
  constexpr int FW = (FR + 3) / 4;             // per warp
  __shared__ __align__(16) __nv_bfloat16 sIn[kHalo * CS];
  __shared__ __align__(16) __nv_bfloat16 sDy[TZ * TY * TX * DS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tap_row = blockIdx.y;  // kz * 3 + ky
  float acc[FW][4];
#pragma unroll
  for (int f = 0; f < FW; ++f)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[f][k] = 0.0f;

  const int tiles_x = W / TX, tiles_y = H / TY, tiles_z = D / TZ;
  const int ntiles = B * tiles_z * tiles_y * tiles_x;
  for (int t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const int tx = t % tiles_x, ty = (t / tiles_x) % tiles_y, tz = (t / (tiles_x * tiles_y)) % tiles_z;
    const int b = t / (tiles_x * tiles_y * tiles_z);
    const int oz = tz * TZ, oy = ty * TY, ox = tx * TX;
    __syncthreads();
    stage_tile<CIN, CS>(sIn, x, b, oz, oy, ox, D, H, W);
    for (int i = threadIdx.x; i < TZ * TY * TX * (COUT / 8); i += kThreads) {
      const int v = i / (COUT / 8), c = i % (COUT / 8);
      const int z = v / (TY * TX), yy = (v / TX) % TY, xx = v % TX;
      *reinterpret_cast<uint4*>(sDy + v * DS + c * 8) = *reinterpret_cast<const uint4*>(
          dy + ((((int64_t)b * D + oz + z) * H + oy + yy) * W + ox + xx) * COUT + c * 8);
    }
    __syncthreads();
    // K = 128 voxels in 8 slices of 16
#pragma unroll
    for (int f = 0; f < FW; ++f) {
      const int fr = warp + 4 * f;
      if (fr >= FR) break;
      const int kx = fr / (MT * NT), mt = (fr / NT) % MT, nt = fr % NT;
      const int dz = tap_row / 3, dyy = tap_row % 3;
#pragma unroll 2
      for (int ks = 0; ks < 8; ++ks) {
        unsigned a0, a1, a2, a3, b0, b1, bx0, bx1;
        // A = dy^T (16 c_out x 16 voxels): stored [voxel][c_out] -> ldmatrix.trans
        {
          const int j = lane >> 3;
          const int v = ks * 16 + (j >> 1) * 8 + (lane & 7);
          const int co = mt * 16 + (j & 1) * 8;
          ldsm_x4_t(smem_u32(sDy + v * DS + co), a0, a1, a2, a3);
        }
        // B = x shifted (16 voxels x 8 c_in): stored [voxel][c_in] -> ldmatrix.trans
        {
          const int j = (lane >> 3) & 1;
          const int v = ks * 16 + j * 8 + (lane & 7);
          ldsm_x4_t(smem_u32(sIn + halo_index(v, dz, dyy, kx) * CS + nt * 8), b0, b1, bx0, bx1);
        }
        mma_bf16(acc[f], a0, a1, a2, a3, b0, b1);
      }
    }
  }
  // write this block's partial sums
  const int g = lane >> 2, tig = lane & 3;
  const int blk = blockIdx.x;
#pragma unroll
  for (int f = 0; f < FW; ++f) {
    const int fr = warp + 4 * f;
    if (fr >= FR) break;
    const int kx = fr / (MT * NT), mt = (fr / NT) % MT, nt = fr % NT;
    const int tap = tap_row * 3 + kx;
    float* dst = part + ((int64_t)blk * 27 + tap) * COUT * CIN;
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int co = mt * 16 + half * 8 + g, ci = nt * 8 + 2 * tig;
      dst[co * CIN + ci] = acc[f][2 * half];
      dst[co * CIN + ci + 1] = acc[f][2 * half + 1];
    }
  }
}

// out[i] = sum_b part[b][i]  (fixed order)
__global__ void k_sum_parts(const float* __restrict__ part, int nb, int64_t n, float* out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int b = 0; b < nb; ++b) s += part[(int64_t)b * n + i];
    out[i] = s;
  }
}

// Bias gradient db[c] = sum over voxels of dy[v][c], in two fixed-order passes.
// Pass 1: block b owns a contiguous range of voxels; a thread owns one 8-channel
// chunk and strides over the range's voxels with 16-byte loads (four loads in
// flight), then the threads of each chunk are summed through shared memory
// into part[b][c].  Pass 2: one thread per channel sums the blocks in order.
template <int C>
__global__ void __launch_bounds__(256) k_bias_part(const __nv_bfloat16* __restrict__ dy,
                                                   int64_t nvox, float* __restrict__ part) {
  constexpr int NC = C / 8, VPI = 256 / NC;  // chunks per voxel, voxels per pass of the block
  __shared__ float red[256 * 9];
  const int c = threadIdx.x % NC, vl = threadIdx.x / NC;
  const int64_t per = (nvox + gridDim.x - 1) / gridDim.x;
  const int64_t v0 = (int64_t)blockIdx.x * per;
  const int64_t v1 = v0 + per < nvox ? v0 + per : nvox;
  float s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
  int64_t v = v0 + vl;
  for (; v + 3 * VPI < v1; v += 4 * VPI) {
    uint4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u)
      q[u] = *reinterpret_cast<const uint4*>(dy + (v + u * VPI) * C + 8 * c);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q[u]);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        s[2 * j] += f.x;
        s[2 * j + 1] += f.y;
      }
    }
  }
  for (; v < v1; v += VPI) {
    const uint4 q = *reinterpret_cast<const uint4*>(dy + v * C + 8 * c);
    const __nv_bfloat162* h = reinterpret_cast<const __nv_bfloat162*>(&q);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 f = __bfloat1622float2(h[j]);
      s[2 * j] += f.x;
      s[2 * j + 1] += f.y;
    }
  }
#pragma unroll
  for (int j = 0; j < 8; ++j) red[threadIdx.x * 9 + j] = s[j];
  __syncthreads();
  if (threadIdx.x < C) {
    const int ch = threadIdx.x, k = ch / 8, j = ch % 8;
    float t = 0.0f;
    for (int r = 0; r < VPI; ++r) t += red[(r * NC + k) * 9 + j];
    part[(int64_t)blockIdx.x * C + ch] = t;
  }
}

// 8 threads per channel each sum every 8th block, then the 8 sums are added in
// a fixed order (deterministic for a given block count).
__global__ void __launch_bounds__(256) k_bias_final(const float* __restrict__ part, int nblk,
                                                    int C, float* db) {
  __shared__ float red[256];
  const int c = threadIdx.x >> 3, k = threadIdx.x & 7;
  float t = 0.0f;
  if (c < C)
    for (int b = k; b < nblk; b += 8) t += part[(int64_t)b * C + c];
  red[threadIdx.x] = t;
  __syncthreads();
  if (k == 0 && c < C) {
    float s = 0.0f;
#pragma unroll
    for (int j = 0; j < 8; ++j) s += red[threadIdx.x + j];
    db[c] = s;
  }
}

}  // namespace

template <int CIN, int COUT>
static cudaError_t conv_launch(const __nv_bfloat16* x, const __nv_bfloat16* wt, const float* bias,
                               int relu, __nv_bfloat16* y16, float* y32, int B, int D, int H, int W,
                               int grid, cudaStream_t s) {
  const int smem = (27 * COUT * (CIN + 8) + kHalo * (CIN + 8)) * 2;
  static std::atomic<unsigned long long> raised{0};
  const cudaError_t e = raise_smem_limit(k_conv3d<CIN, COUT>, smem, raised);
  if (e != cudaSuccess) return e;
  const int ntiles = B * (D / TZ) * (H / TY) * (W / TX);
  k_conv3d<CIN, COUT><<<grid < ntiles ? grid : ntiles, kThreads, smem, s>>>(x, wt, bias, relu, y16,
                                                                          y32, B, D, H, W);
  return cudaGetLastError();
}

cudaError_t launch_conv3d(int cin, int cout, const void* x, const void* wt, const float* bias,
                          int relu, void* y16, float* y32, int B, int D, int H, int W, int grid,
                          cudaStream_t s) {
  const __nv_bfloat16* X = (const __nv_bfloat16*)x;
  const __nv_bfloat16* Wt = (const __nv_bfloat16*)wt;
  __nv_bfloat16* Y = (__nv_bfloat16*)y16;
  if (cin == 16 && cout == 32) return conv_launch<16, 32>(X, Wt, bias, relu, Y, y32, B, D, H, W, grid, s);
  if (cin == 32 && cout == 32) return conv_launch<32, 32>(X, Wt, bias, relu, Y, y32, B, D, H, W, grid, s);
  if (cin == 32 && cout == 16) return conv_launch<32, 16>(X, Wt, bias, relu, Y, y32, B, D, H, W, grid, s);
  return cudaErrorInvalidValue;
}

int conv_wgrad_blocks(int B, int D, int H, int W, int max_blocks) {
  const int ntiles = B * (D / TZ) * (H / TY) * (W / TX);
  return ntiles < max_blocks ? ntiles : max_blocks;
}

cudaError_t launch_conv3d_wgrad(int cin, int cout, const void* x, const void* dy, float* part,
                                float* dw, int B, int D, int H, int W, int blocks, cudaStream_t s) {
  const __nv_bfloat16* X = (const __nv_bfloat16*)x;
  const __nv_bfloat16* DY = (const __nv_bfloat16*)dy;
  const dim3 grid(blocks, 9);
  if (cin == 16 && cout == 32)
    k_conv3d_wgrad<16, 32><<<grid, kThreads, 0, s>>>(X, DY, part, B, D, H, W);
  else if (cin == 32 && cout == 32)
    k_conv3d_wgrad<32, 32><<<grid, kThreads, 0, s>>>(X, DY, part, B, D, H, W);
  else if (cin == 32 && cout == 16)
    k_conv3d_wgrad<32, 16><<<grid, kThreads, 0, s>>>(X, DY, part, B, D, H, W);
  else
    return cudaErrorInvalidValue;
  const int64_t n = (int64_t)27 * cin * cout;
  k_sum_parts<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(part, blocks, n, dw);
  return cudaGetLastError();
}

int bias_grad_blocks() { return 4 * device_sm_count(); }

cudaError_t launch_bias_grad(const void* dy, int C, int64_t nvox, float* db, float* scratch,
                             cudaStream_t s) {
  const __nv_bfloat16* DY = (const __nv_bfloat16*)dy;
  int64_t nb = bias_grad_blocks();
  if (nb > nvox) nb = nvox < 1 ? 1 : nvox;
  if (C == 16)
    k_bias_part<16><<<(unsigned)nb, 256, 0, s>>>(DY, nvox, scratch);
  else if (C == 32)
    k_bias_part<32><<<(unsigned)nb, 256, 0, s>>>(DY, nvox, scratch);
  else
    return cudaErrorInvalidValue;
  k_bias_final<<<1, 256, 0, s>>>(scratch, (int)nb, C, db);  // C <= 32
  return cudaGetLastError();
}

}  // namespace pf
