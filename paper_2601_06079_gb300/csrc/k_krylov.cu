// Vector kernels of the Newton-GMRES solver (JAX-PF Eq. 13-14).  The Krylov
// basis is FP32; every inner product and norm keeps about 48 bits per thread
// and finishes in FP64: each thread forms FP32 sums over 8 consecutive
// products and adds them into a compensated FP32 pair (hi + lo, Knuth's
// two-sum), warps combine the pairs the same way and blocks add the warps'
// values in FP64, and the last block sums the per-block partials in a fixed
// order, so results are deterministic.  No FP64 arithmetic runs per element: GB300 issues about 2
// FP64 operations per clock per SM, 64 times fewer than FP32.
#include "pf_internal.h"

namespace pf {
namespace {

constexpr int kThreads = 256;
constexpr int kChunk = 8;      // products per FP32 partial sum
constexpr int kMaxFields = 8;  // order parameters of a Newton vector (planes of the mass norm)

// s added to the unevaluated sum hi + lo (Knuth's two-sum: the rounding error
// of hi + s is exact in FP32 and collects in lo)
struct Acc2 {
  float hi = 0.0f, lo = 0.0f;
  __device__ __forceinline__ void add(float s) {
    const float t = hi + s;
    const float bp = t - hi;
    lo += (hi - (t - bp)) + (s - bp);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

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

// Block-wide sum of the threads' compensated pairs, valid in thread 0: the
// warp tree combines pairs in FP32 (two-sum, the low parts added), only the
// warps' values are summed in FP64 (a tree in warp 0), in a fixed order.
__device__ double block_sum2(Acc2 a, double* scratch) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h = __shfl_down_sync(0xffffffffu, a.hi, o);
    const float l = __shfl_down_sync(0xffffffffu, a.lo, o);
    a.add(h);
    a.lo += l;
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) scratch[w] = a.value();
  __syncthreads();
  double v = 0.0;
  if (w == 0) {
    v = l < kThreads / 32 ? scratch[l] : 0.0;
#pragma unroll
    for (int o = kThreads / 64; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  }
  return v;
}

// The last block to finish sums all blocks' partials[b * k + j] into out[j]
// in the fixed order of a separate single-block pass (b ascending per thread,
// then the block sum), so one launch gives the final, repeatable values.
// count: device counter, 0 before the launch and reset to 0 by the last block.
__device__ void finish_sum(const double* partials, int k, double* __restrict__ out,
                           unsigned* count, double* scratch) {
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(count, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int j = 0; j < k; ++j) {
    double acc = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) acc += __ldcg(partials + b * k + j);
    acc = block_sum(acc, scratch);
    if (threadIdx.x == 0) out[j] = acc;
  }
  if (threadIdx.x == 0) *count = 0;
}

// Chunks of kChunk = 8 consecutive values: two 16-byte loads when the vectors
// are 16-byte aligned (kVec) and the chunk is whole, elementwise otherwise
// (values past n read as 0).  Each kernel below is instantiated for a bound
// KMAX on the number of basis vectors (4, 8, 16, 32), so that its accumulators
// (compensated FP32 pairs) take registers only for the vectors a call can have.
template <bool kVec>
__device__ __forceinline__ void load8(const float* __restrict__ p, int64_t i0, int64_t n,
                                      float v[kChunk]) {
  if (kVec && i0 + kChunk <= n) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p + i0));
    const float4 b = __ldg(reinterpret_cast<const float4*>(p + i0 + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int t = 0; t < kChunk; ++t) v[t] = (i0 + t < n) ? p[i0 + t] : 0.0f;
  }
}

// load8 through L2 only (ld.global.cg): for values this kernel wrote itself,
// which the non-coherent read-only path of load8 may not see
template <bool kVec>
__device__ __forceinline__ void load8_cg(const float* p, int64_t i0, int64_t n, float v[kChunk]) {
  if (kVec && i0 + kChunk <= n) {
    const float4 a = __ldcg(reinterpret_cast<const float4*>(p + i0));
    const float4 b = __ldcg(reinterpret_cast<const float4*>(p + i0 + 4));
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
  } else {
#pragma unroll
    for (int t = 0; t < kChunk; ++t) v[t] = (i0 + t < n) ? __ldcg(p + i0 + t) : 0.0f;
  }
}

template <bool kVec>
__device__ __forceinline__ void store8(float* __restrict__ p, int64_t i0, int64_t n,
                                       const float v[kChunk]) {
  if (kVec && i0 + kChunk <= n) {
    *reinterpret_cast<float4*>(p + i0) = make_float4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<float4*>(p + i0 + 4) = make_float4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int t = 0; t < kChunk; ++t)
      if (i0 + t < n) p[i0 + t] = v[t];
  }
}

// FP32 run of the chunk's products u[t] v[t], t in order (values past n skipped)
__device__ __forceinline__ float chunk_dot(const float v[kChunk], const float u[kChunk],
                                           int64_t i0, int64_t n) {
  float s = 0.0f;
#pragma unroll
  for (int t = 0; t < kChunk; ++t)
    if (i0 + t < n) s = fmaf(v[t], u[t], s);
  return s;
}

// Block sums of the accumulators of vectors j0 .. j0 + G - 1 (those below k)
// into partials[blockIdx.x * k + j].
template <int G>
__device__ __forceinline__ void group_partials(Acc2 (&acc)[G], int j0, int k, double* scratch,
                                               double* partials) {
#pragma unroll
  for (int j = 0; j < G; ++j) {
    if (j0 + j < k) {
      const double r = block_sum2(acc[j], scratch);
      if (threadIdx.x == 0) partials[blockIdx.x * k + j0 + j] = r;
    }
  }
}

// Inner products take the basis vectors in groups per pass over the chunks
// (w re-read per group; kGroupDots in k_dots, which holds two chunks per
// vector in flight, kGroup in the fused k_update_dots): each j's per-thread
// sum still runs over the same chunks in the same order, so the results do
// not depend on the grouping, and the accumulators (2 registers per vector)
// stay within the 80 registers a thread may hold at 3 blocks of 256 threads
// per SM, the residency that the fixed grid of 3 blocks per SM needs to run
// in one wave.
constexpr int kGroup = 16;
constexpr int kGroupDots = 8;
constexpr int kMinBlocks = 3;

// out[j] = V_j . w (j < k <= KMAX), V_j = V + j * ldv; w is read once per
// group of kGroupDots products (per-block partials in `partials`).  If
// w == nullptr the squared norm of V_0 is taken (k must be 1).
template <int KMAX, bool kVec>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_dots(const float* __restrict__ V,
                                                               int64_t ldv, int k,
                                                               const float* __restrict__ w,
                                                               int64_t n, double* partials,
                                                               double* out, unsigned* count) {
  constexpr int G = KMAX < kGroupDots ? KMAX : kGroupDots;
  __shared__ double scratch[kThreads / 32];
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  const float* x = w ? w : V;
  for (int j0 = 0; j0 < k; j0 += G) {
    Acc2 acc[G];
    // two of the thread's chunks per iteration (twice the loads in flight),
    // added in chunk order
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks; c += 2 * stride) {
      const int64_t i0 = c * kChunk, i1 = (c + stride) * kChunk;
      const bool second = c + stride < chunks;
      float u0[kChunk], u1[kChunk];
      load8<kVec>(x, i0, n, u0);
      if (second) load8<kVec>(x, i1, n, u1);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j0 + j < k) {
          float v0[kChunk], v1[kChunk];
          load8<kVec>(V + (j0 + j) * ldv, i0, n, v0);
          if (second) load8<kVec>(V + (j0 + j) * ldv, i1, n, v1);
          acc[j].add(chunk_dot(v0, u0, i0, n));
          if (second) acc[j].add(chunk_dot(v1, u1, i1, n));
        }
      }
    }
    group_partials<G>(acc, j0, k, scratch, partials);
  }
  finish_sum(partials, k, out, count, scratch);
}

// x <- x - sum_j cf[j] V_j over one chunk, j in order for every element
template <int KMAX, bool kVec>
__device__ __forceinline__ void chunk_update(const float* __restrict__ V, int64_t ldv, int k,
                                             const float* cf, int64_t i0, int64_t n,
                                             float x[kChunk]) {
  // up to 8 vectors fully unrolled; beyond, groups of 4 (a full unroll of 16
  // or 32 hoists every vector's loads and takes up to 255 registers)
#pragma unroll(KMAX <= 8 ? KMAX : 4)
  for (int j = 0; j < k; ++j) {
    float v[kChunk];
    load8<kVec>(V + j * ldv, i0, n, v);
#pragma unroll
    for (int t = 0; t < kChunk; ++t) x[t] = fmaf(-cf[j], v[t], x[t]);
  }
}

// w <- w - sum_j coef[j] V_j (coef: device FP64);  optionally (norm_out) |w|^2
template <int KMAX, bool kVec>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_update(const float* __restrict__ V,
                                                                 int64_t ldv, int k,
                                                                 const double* __restrict__ coef,
                                                                 float* __restrict__ w, int64_t n,
                                                                 double* partials,
                                                                 double* norm_out,
                                                                 unsigned* count) {
  __shared__ double scratch[kThreads / 32];
  __shared__ float cf[KMAX];
  for (int j = threadIdx.x; j < k; j += kThreads) cf[j] = (float)coef[j];
  __syncthreads();
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  Acc2 acc;
  // two of the thread's chunks per iteration (twice the loads in flight); each
  // element's update and the norm's chunk order are those of one at a time
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks; c += 2 * stride) {
    const int64_t i0 = c * kChunk, i1 = (c + stride) * kChunk;
    const bool second = c + stride < chunks;
    float x0[kChunk], x1[kChunk];
    load8<kVec>(w, i0, n, x0);
    if (second) load8<kVec>(w, i1, n, x1);
#pragma unroll(KMAX <= 4 ? KMAX : 2)
    for (int j = 0; j < k; ++j) {
      float v0[kChunk], v1[kChunk];
      load8<kVec>(V + j * ldv, i0, n, v0);
      if (second) load8<kVec>(V + j * ldv, i1, n, v1);
#pragma unroll
      for (int t = 0; t < kChunk; ++t) {
        x0[t] = fmaf(-cf[j], v0[t], x0[t]);
        if (second) x1[t] = fmaf(-cf[j], v1[t], x1[t]);
      }
    }
    store8<kVec>(w, i0, n, x0);
    if (second) store8<kVec>(w, i1, n, x1);
    if (norm_out) {
      acc.add(chunk_dot(x0, x0, i0, n));
      if (second) acc.add(chunk_dot(x1, x1, i1, n));
    }
  }
  if (norm_out) {
    const double r = block_sum2(acc, scratch);
    if (threadIdx.x == 0) partials[blockIdx.x] = r;
    finish_sum(partials, 1, norm_out, count, scratch);
  }
}

// w <- w - sum_j coef[j] V_j, and partials[b * k + j] of V_j . w for the
// updated w: the two halves of a CGS2 pass boundary (the first pass's update
// and the second pass's inner products) in one pass over V and w.  Each
// element's arithmetic and each thread's chunks are those of k_update
// followed by k_dots, so the results are identical to the two kernels.  The
// pass takes the products of the first kGroup vectors; later groups re-read
// the updated w (this thread's own stores, through L2) and their vectors.
template <int KMAX, bool kVec>
__global__ void __launch_bounds__(kThreads, kMinBlocks) k_update_dots(
    const float* __restrict__ V, int64_t ldv, int k, const double* __restrict__ coef,
    float* __restrict__ w, int64_t n, double* partials, double* out, unsigned* count) {
  constexpr int G = KMAX < kGroup ? KMAX : kGroup;
  __shared__ double scratch[kThreads / 32];
  __shared__ float cf[KMAX];
  for (int j = threadIdx.x; j < k; j += kThreads) cf[j] = (float)coef[j];
  __syncthreads();
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  {
    Acc2 acc[G];
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * kThreads) {
      const int64_t i0 = c * kChunk;
      float x[kChunk];
      load8<kVec>(w, i0, n, x);
      chunk_update<KMAX, kVec>(V, ldv, k, cf, i0, n, x);
      store8<kVec>(w, i0, n, x);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j < k) {
          float v[kChunk];
          load8<kVec>(V + j * ldv, i0, n, v);
          acc[j].add(chunk_dot(v, x, i0, n));
        }
      }
    }
    group_partials<G>(acc, 0, k, scratch, partials);
  }
  for (int j0 = G; j0 < k; j0 += G) {
    Acc2 acc[G];
    for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks;
         c += (int64_t)gridDim.x * kThreads) {
      const int64_t i0 = c * kChunk;
      float x[kChunk];
      load8_cg<kVec>(w, i0, n, x);
#pragma unroll
      for (int j = 0; j < G; ++j) {
        if (j0 + j < k) {
          float v[kChunk];
          load8<kVec>(V + (j0 + j) * ldv, i0, n, v);
          acc[j].add(chunk_dot(v, x, i0, n));
        }
      }
    }
    group_partials<G>(acc, j0, k, scratch, partials);
  }
  finish_sum(partials, k, out, count, scratch);
}

// y <- a * x + b * y  (host scalars), chunks of 8
template <bool kVec>
__global__ void k_axpby(float a, const float* __restrict__ x, float b, float* __restrict__ y,
                        int64_t n) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = c * kChunk;
    float u[kChunk], v[kChunk];
    load8<kVec>(x, i0, n, u);
    load8<kVec>(y, i0, n, v);
#pragma unroll
    for (int t = 0; t < kChunk; ++t) v[t] = fmaf(a, u[t], b * v[t]);
    store8<kVec>(y, i0, n, v);
  }
}

// x <- x + sum_j y_j V_j, j in order for every element, chunks of 8
template <int KMAX, bool kVec>
__global__ void k_lincomb(const float* __restrict__ V, int64_t ldv, int k, LinComb y,
                          float* __restrict__ x, int64_t n) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < chunks;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i0 = c * kChunk;
    float s[kChunk];
    load8<kVec>(x, i0, n, s);
#pragma unroll
    for (int j = 0; j < KMAX; ++j) {
      if (j < k) {
        float v[kChunk];
        load8<kVec>(V + j * ldv, i0, n, v);
#pragma unroll
        for (int t = 0; t < kChunk; ++t) s[t] = fmaf(y.c[j], v[t], s[t]);
      }
    }
    store8<kVec>(x, i0, n, s);
  }
}

// lumped-mass boundary factor: 1/2 per axis on which the node is an end node
// (nz = 1 is a 2-D mesh)
__device__ __forceinline__ float mass_factor(int x, int y, int z, int nx, int ny, int nz) {
  float m = 1.0f;
  if (x == 0 || x == nx - 1) m *= 0.5f;
  if (y == 0 || y == ny - 1) m *= 0.5f;
  if (nz > 1 && (z == 0 || z == nz - 1)) m *= 0.5f;
  return m;
}

// sum_i (m_i g_i)^2 over all fields into out[0]: m_i = cell * boundary factor.
// Each thread takes chunks of 4 consecutive nodes (one index division per
// chunk; kVec: one 16-byte load per field when the node count is a multiple
// of 4).  Products in FP32 (GB300's FP64 rate is a small fraction of its FP32
// rate), a chunk's squares summed in FP32, the chunks in a compensated FP32
// pair, the block sums in FP64.
template <bool kVec>
__global__ void __launch_bounds__(kThreads) k_mass_norm(const float* __restrict__ g, int nx,
                                                        int ny, int nz, int nf, float cell,
                                                        double* partials, double* out,
                                                        unsigned* count) {
  __shared__ double scratch[kThreads / 32];
  const int64_t N = (int64_t)nx * ny * nz;
  const int64_t chunks = (N + 3) / 4;
  Acc2 acc;
  for (int64_t c = (int64_t)blockIdx.x * kThreads + threadIdx.x; c < chunks;
       c += (int64_t)gridDim.x * kThreads) {
    const int64_t i0 = 4 * c;
    // node coordinates in 32-bit arithmetic (nodes < 2^31): a 64-bit integer
    // division runs on the FP64 pipe, a small fraction of GB300's FP32 rate
    const int node0 = (int)i0;
    int x = node0 % nx;
    const int r = node0 / nx;
    int y = r % ny, z = r / ny;
    float m[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      m[t] = (i0 + t < N) ? cell * mass_factor(x, y, z, nx, ny, nz) : 0.0f;
      if (++x == nx) {
        x = 0;
        if (++y == ny) {
          y = 0;
          ++z;
        }
      }
    }
    // every field's chunk is loaded before any is used, so the loads of up
    // to kMaxFields planes are in flight together
    float v[kMaxFields][4];
#pragma unroll
    for (int f = 0; f < kMaxFields; ++f) {
      if (f < nf) {
        const float* p = g + (int64_t)f * N + i0;
        if (kVec && i0 + 4 <= N) {
          const float4 q = __ldg(reinterpret_cast<const float4*>(p));
          v[f][0] = q.x; v[f][1] = q.y; v[f][2] = q.z; v[f][3] = q.w;
        } else {
#pragma unroll
          for (int t = 0; t < 4; ++t) v[f][t] = (i0 + t < N) ? p[t] : 0.0f;
        }
      }
    }
    // the chunk's squares (at most 32) as one FP32 run, then one FP64 add
    float run = 0.0f;
#pragma unroll
    for (int f = 0; f < kMaxFields; ++f) {
      if (f < nf) {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float u = m[t] * v[f][t];
          run = fmaf(u, u, run);
        }
      }
    }
    acc.add(run);
  }
  const double r = block_sum2(acc, scratch);
  if (threadIdx.x == 0) partials[blockIdx.x] = r;
  finish_sum(partials, 1, out, count, scratch);
}

// out = a * m_i^(+1 or -1) * in over nf planes of nx x ny x nz nodes, m the
// lumped mass (cell times 1/2 per boundary axis; nz = 1 is a 2-D mesh);
// inv_cell = 1 / cell, so that the inverse is a multiplication
__global__ void k_mass_mul(const float* __restrict__ in, float* __restrict__ out, int nx, int ny,
                           int nz, int nf, float cell, float inv_cell, float a, int inverse) {
  const int N = nx * ny * nz;
  for (int node = blockIdx.x * blockDim.x + threadIdx.x; node < N; node += gridDim.x * blockDim.x) {
    const float fac = mass_factor(node % nx, (node / nx) % ny, node / (nx * ny), nx, ny, nz);
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

namespace {
// 16-byte loads when every vector the call touches starts on a 16-byte boundary
bool vec_ok(const void* a, const void* b, int64_t ldv) {
  return ((uintptr_t)a % 16 == 0) && ((uintptr_t)b % 16 == 0) && (ldv % 4 == 0);
}

// calls K<KMAX, kVec> for the smallest KMAX in {4, 8, 16, 32} holding k
template <template <int, bool> class K, typename... A>
cudaError_t dispatch_k(int k, bool vec, cudaStream_t s, A... args) {
  const dim3 g(krylov_partial_blocks()), b(kThreads);
#define PF_KRYLOV_CASE(M)                                            \
  if (k <= M) {                                                      \
    if (vec) K<M, true>::launch(g, b, s, args...);                   \
    else K<M, false>::launch(g, b, s, args...);                      \
    return cudaGetLastError();                                       \
  }
  PF_KRYLOV_CASE(4)
  PF_KRYLOV_CASE(8)
  PF_KRYLOV_CASE(16)
  PF_KRYLOV_CASE(kMaxBasis)
#undef PF_KRYLOV_CASE
  return cudaErrorInvalidValue;
}

template <int M, bool V>
struct Dots {
  template <typename... A>
  static void launch(dim3 g, dim3 b, cudaStream_t s, A... a) { k_dots<M, V><<<g, b, 0, s>>>(a...); }
};
template <int M, bool V>
struct Update {
  template <typename... A>
  static void launch(dim3 g, dim3 b, cudaStream_t s, A... a) { k_update<M, V><<<g, b, 0, s>>>(a...); }
};
template <int M, bool V>
struct UpdateDots {
  template <typename... A>
  static void launch(dim3 g, dim3 b, cudaStream_t s, A... a) {
    k_update_dots<M, V><<<g, b, 0, s>>>(a...);
  }
};
}  // namespace

cudaError_t launch_dots(const float* V, int64_t ldv, int k, const float* w, int64_t n,
                        double* partials, double* out, unsigned* count, cudaStream_t s) {
  return dispatch_k<Dots>(k, vec_ok(V, w ? w : V, ldv), s, V, ldv, k, w, n, partials, out, count);
}

cudaError_t launch_update(const float* V, int64_t ldv, int k, const double* coef, float* w,
                          int64_t n, double* partials, double* norm_out, unsigned* count,
                          cudaStream_t s) {
  return dispatch_k<Update>(k, vec_ok(V, w, ldv), s, V, ldv, k, coef, w, n, partials, norm_out,
                            count);
}

cudaError_t launch_update_dots(const float* V, int64_t ldv, int k, const double* coef, float* w,
                               int64_t n, double* partials, double* out, unsigned* count,
                               cudaStream_t s) {
  return dispatch_k<UpdateDots>(k, vec_ok(V, w, ldv), s, V, ldv, k, coef, w, n, partials, out,
                                count);
}

cudaError_t launch_axpby(float a, const float* x, float b, float* y, int64_t n, cudaStream_t s) {
  const unsigned g = elementwise_blocks((n + kChunk - 1) / kChunk);
  if (vec_ok(x, y, 0))
    k_axpby<true><<<g, 256, 0, s>>>(a, x, b, y, n);
  else
    k_axpby<false><<<g, 256, 0, s>>>(a, x, b, y, n);
  return cudaGetLastError();
}

cudaError_t launch_lincomb(const float* V, int64_t ldv, int k, const LinComb& y, float* x,
                           int64_t n, cudaStream_t s) {
  const dim3 g(elementwise_blocks((n + kChunk - 1) / kChunk)), b(256);
  const bool vec = vec_ok(V, x, ldv);
#define PF_LINCOMB_CASE(M)                                                  \
  if (k <= M) {                                                             \
    if (vec) k_lincomb<M, true><<<g, b, 0, s>>>(V, ldv, k, y, x, n);        \
    else k_lincomb<M, false><<<g, b, 0, s>>>(V, ldv, k, y, x, n);           \
    return cudaGetLastError();                                              \
  }
  PF_LINCOMB_CASE(4)
  PF_LINCOMB_CASE(8)
  PF_LINCOMB_CASE(16)
  PF_LINCOMB_CASE(kMaxBasis)
#undef PF_LINCOMB_CASE
  return cudaErrorInvalidValue;
}

cudaError_t launch_mass_mul(const float* in, float* out, int nx, int ny, int nz, int nf,
                            double cell, float a, int inverse, cudaStream_t s) {
  k_mass_mul<<<elementwise_blocks((int64_t)nx * ny * nz), 256, 0, s>>>(
      in, out, nx, ny, nz, nf, (float)cell, (float)(1.0 / cell), a, inverse);
  return cudaGetLastError();
}

cudaError_t launch_mass_norm(const float* g, int nx, int ny, int nz, int nf, double cell,
                             double* partials, double* out, unsigned* count, cudaStream_t s) {
  const int64_t N = (int64_t)nx * ny * nz;
  if (nf < 1 || nf > kMaxFields) return cudaErrorInvalidValue;
  if (N % 4 == 0 && (uintptr_t)g % 16 == 0)
    k_mass_norm<true><<<krylov_partial_blocks(), kThreads, 0, s>>>(g, nx, ny, nz, nf, (float)cell,
                                                                    partials, out, count);
  else
    k_mass_norm<false><<<krylov_partial_blocks(), kThreads, 0, s>>>(g, nx, ny, nz, nf, (float)cell,
                                                                     partials, out, count);
  return cudaGetLastError();
}

}  // namespace pf
