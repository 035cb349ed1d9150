// Fused 2-D explicit step kernels: element gather -> Gauss-point values ->
// f'(u_q) -> node-centric gather of the element contributions -> gradient
// stencil -> lumped-mass Euler update (JAX-PF Eq. 11-12; Cahn-Hilliard via the
// split form of Eq. 9-10).  One pass reads the state once and writes it once.
//
// Work split.  A warp owns 64 consecutive columns (a pair per lane) and
// sweeps down a band of rows with a sliding window in registers; the
// neighbouring columns come from the adjacent lanes by warp shuffle, so there
// is no shared memory and no block barrier, and every element is evaluated
// once per warp.  Lanes 0 and 31 are halo lanes (their outer column lacks a
// neighbour), so warps overlap by 4 columns and each writes the 60 columns of
// lanes 1..30.  All arithmetic is on packed FP32 pairs (one lane's two
// columns) with the f32x2 instructions of sm_100+, which halve the issue slots
// of the FP32 work.
//
// Quadrature is sum-factorised: per row, two x-interpolated values per
// segment; per element, the four Gauss values from the segment values of its
// two rows; the weights N_a(q) are applied back the same way (y first into
// per-segment sums, then x into the nodes).  Interpolation uses
// g_hi = 1 - g_lo, e.g. g_hi a + g_lo b = a + g_lo (b - a).  The linear
// gradient term is the exact assembled 9-point Q1 stencil (2x2 Gauss
// integrates it exactly); on square cells it is a v + b (sum of the 3x3 block).
// Zero-flux boundaries are the mirror extension about the boundary nodes,
// which equals the partial element sets divided by the partial lumped masses
// (both double when mirrored), so every node uses the interior formula.  The
// working planes carry that extension explicitly: a frame of 2 ghost rows and
// columns that every step rewrites from the nodes it mirrors, so all warps run
// the same branch-free sweep with no index reflection.
#include <string.h>

#include "pf_internal.h"

namespace pf {
namespace {

typedef unsigned long long u64;  // packed FP32 pair: low half = lower column

constexpr int kPair = 2;                          // columns per lane
constexpr int kOutCols = 32 * kPair - 2 * kPair;  // 60 output columns per warp
#ifndef PF_WARPS
#define PF_WARPS 2
#endif
constexpr int kWarps = PF_WARPS;                  // warps per block, stacked in y
constexpr unsigned kFull = 0xffffffffu;
constexpr int kGhost = 2;  // mirror frame around the working planes
#ifndef PF_ROWS_AHEAD
#define PF_ROWS_AHEAD 6
#endif
#ifndef PF_MINB
#define PF_MINB 1  // minimum resident blocks per SM asked of the register allocator
#endif
#ifndef PF_ENS_MINB
#define PF_ENS_MINB 6  // minimum resident ensemble blocks per SM asked of the register allocator
#endif
#ifndef PF_ENS_COEF
#define PF_ENS_COEF 2  // ensemble coefficients: 0 registers, 1 instance table, 2 shared memory
#endif
#ifndef PF_PDL
#define PF_PDL 0  // 1: programmatic dependent launch, dependents released at block end
#endif
constexpr int kAhead = PF_ROWS_AHEAD;  // rows loaded ahead of use (divides the unroll of 6)

__device__ __forceinline__ u64 pk(float lo, float hi) {
  u64 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float plo(u64 v) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(v));
  return l;
}
__device__ __forceinline__ float phi(u64 v) {
  float l, h;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(l), "=f"(h) : "l"(v));
  return h;
}
__device__ __forceinline__ u64 fma2(u64 a, u64 b, u64 c) {
  u64 d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ u64 add2(u64 a, u64 b) {
  u64 d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 sub2(u64 a, u64 b) {
  u64 d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 mul2(u64 a, u64 b) {
  u64 d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ u64 bc(float v) { return pk(v, v); }

__device__ __forceinline__ int reflect_row(int k, int n) {
  k = k < 0 ? -k : k;
  k = k >= n ? 2 * (n - 1) - k : k;
  return k < 0 ? 0 : (k >= n ? n - 1 : k);  // rows this far out are never stored
}

__device__ __forceinline__ int reflect_col(int x, int n) {
  const int p = 2 * (n - 1);
  x %= p;
  if (x < 0) x += p;
  return x < n ? x : p - x;
}

// f'(shift + d) / 4 (times the stage factor) as a cubic in d
__device__ __forceinline__ u64 cubic2(u64 d, u64 p0, u64 p1, u64 p2, u64 p3) {
  return fma2(fma2(fma2(p3, d, p2), d, p1), d, p0);
}

// Packed constants, read straight from the kernel parameter space.
struct Coef {
  const unsigned long long* c;
  __device__ __forceinline__ u64 glo() const { return c[0]; }
  __device__ __forceinline__ u64 ghi() const { return c[1]; }
  __device__ __forceinline__ u64 nglo() const { return c[2]; }
  __device__ __forceinline__ u64 p(int i) const { return c[3 + i]; }
  __device__ __forceinline__ u64 k(int stage, int i) const { return c[7 + 6 * stage + i]; }
};

// Per-row stencil helper value: iso -> v + (v_W + v_E) (3-sum of the row);
// general -> v_W + v_E.
template <bool kIso>
__device__ __forceinline__ u64 row_aux(u64 v, u64 hs) {
  return kIso ? add2(v, hs) : hs;
}

// init + K v at the centre row (own values s/c/n, row helpers aux_s/aux_c/aux_n)
template <bool kIso>
__device__ __forceinline__ u64 stencil2(u64 init, u64 s, u64 c, u64 n, u64 aux_s, u64 aux_c,
                                        u64 aux_n, u64 ka, u64 kb, u64 c0, u64 cx, u64 cy,
                                        u64 cd) {
  if (kIso) {
    const u64 s9 = add2(add2(aux_s, aux_c), aux_n);
    return fma2(kb, s9, fma2(ka, c, init));
  } else {
    return fma2(cd, add2(aux_s, aux_n), fma2(cy, add2(s, n), fma2(cx, aux_c, fma2(c0, c, init))));
  }
}

// Sliding-window state of one lane (rows k-1, k-2, ...).
struct Window {
  u64 c1 = 0, c2 = 0, x1 = 0, x2 = 0;      // own values and row helpers, rows k-1, k-2
  u64 am1 = 0, ap1 = 0;                    // x-interpolants of row k-1
  u64 tl1 = 0, th1 = 0;                    // element row k-2 -> node row k-1
  u64 mua = 0, mub = 0, mxa = 0, mxb = 0;  // CH: mu and helpers, rows k-3, k-2
};

// One row of the sweep: consume row k (P), advance the window, return the
// finished output row (k-1 for AC, k-2 for CH).
template <bool kCH, bool kIso>
__device__ __forceinline__ u64 sweep_row(const u64 P, Window& w, const Coef& K) {
  const float c0 = plo(P), c1v = phi(P);
  const float cl = __shfl_up_sync(kFull, c1v, 1);   // column x-1
  const float cr = __shfl_down_sync(kFull, c0, 1);  // column x+2
  // horizontal neighbour sums and segment differences, formed as scalars so
  // that no pair has to be re-packed from halves of other pairs
  const u64 hs = pk(cl + c1v, c0 + cr);
  const u64 dc = pk(c1v - c0, cr - c1v);
  const u64 xr = row_aux<kIso>(P, hs);

  // x-interpolation of row k on segments x, x+1 at xi = g_lo (am) and g_hi (ap)
  const u64 am = fma2(K.glo(), dc, P);
  const u64 ap = fma2(K.ghi(), dc, P);

  // element row k-1: four Gauss values, f', weights back in y
  const u64 dm = sub2(am, w.am1);
  const u64 dp = sub2(ap, w.ap1);
  const u64 fll = cubic2(fma2(K.glo(), dm, w.am1), K.p(0), K.p(1), K.p(2), K.p(3));
  const u64 flh = cubic2(fma2(K.ghi(), dm, w.am1), K.p(0), K.p(1), K.p(2), K.p(3));
  const u64 fhl = cubic2(fma2(K.glo(), dp, w.ap1), K.p(0), K.p(1), K.p(2), K.p(3));
  const u64 fhh = cubic2(fma2(K.ghi(), dp, w.ap1), K.p(0), K.p(1), K.p(2), K.p(3));
  const u64 dl = sub2(flh, fll);
  const u64 dh = sub2(fhh, fhl);
  const u64 sl = add2(fma2(K.glo(), dl, fll), w.tl1);  // node row k-1, xi = g_lo
  const u64 sh = add2(fma2(K.glo(), dh, fhl), w.th1);  // node row k-1, xi = g_hi
  const u64 tl = fma2(K.nglo(), dl, flh);              // node row k (next row)
  const u64 th = fma2(K.nglo(), dh, fhh);
  // weights back in x: segment s gives A to node s and B to node s+1
  const u64 ds = sub2(sh, sl);
  const u64 A = fma2(K.glo(), ds, sl);
  const u64 B = fma2(K.nglo(), ds, sh);
  const float bl = __shfl_up_sync(kFull, phi(B), 1);
  const u64 F = pk(plo(A) + bl, phi(A) + plo(B));

  u64 o;
  if constexpr (!kCH) {
    // u(k-1) <- u + F + K1 u   (coefficients carry -dt L / m)
    o = stencil2<kIso>(add2(w.c1, F), w.c2, w.c1, P, w.x2, w.x1, xr, K.k(0, 0), K.k(0, 1), K.k(0, 2),
                       K.k(0, 3), K.k(0, 4), K.k(0, 5));
  } else {
    // mu(k-1) = F + K1 c ; then c(k-2) <- c + K2 mu   (K2 carries -dt M / m)
    const u64 mu = stencil2<kIso>(F, w.c2, w.c1, P, w.x2, w.x1, xr, K.k(0, 0), K.k(0, 1), K.k(0, 2),
                                  K.k(0, 3), K.k(0, 4), K.k(0, 5));
    const float m0 = plo(mu), m1 = phi(mu);
    const float ml = __shfl_up_sync(kFull, m1, 1);
    const float mr = __shfl_down_sync(kFull, m0, 1);
    const u64 mx = row_aux<kIso>(mu, pk(ml + m1, m0 + mr));
    o = stencil2<kIso>(w.c2, w.mua, w.mub, mu, w.mxa, w.mxb, mx, K.k(1, 0), K.k(1, 1), K.k(1, 2), K.k(1, 3),
                       K.k(1, 4), K.k(1, 5));
    w.mua = w.mub;
    w.mxa = w.mxb;
    w.mub = mu;
    w.mxb = mx;
  }
  w.c2 = w.c1;
  w.x2 = w.x1;
  w.c1 = P;
  w.x1 = xr;
  w.am1 = am;
  w.ap1 = ap;
  w.tl1 = tl;
  w.th1 = th;
  return o;
}

// Output of one finished pair: real row y, real columns x (lo) and x+1 (hi),
// plus every ghost cell that mirrors it (rows -1, -2 <- 1, 2 and
// ny, ny+1 <- ny-2, ny-3; the same for columns), so the next step reads the
// mirror extension without any index reflection.
__device__ __forceinline__ void store_cols(float* __restrict__ row, int x, int nx, u64 v) {
  const float lo = plo(v), hi = phi(v);
  if (x + 1 < nx) {
    *reinterpret_cast<u64*>(row + x) = v;
  } else {
    row[x] = lo;
  }
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int xc = x + h;
    const float val = h ? hi : lo;
    if (xc >= nx) break;
    if (xc == 1 || xc == 2) row[-xc] = val;
    if (xc == nx - 2 || xc == nx - 3) row[2 * (nx - 1) - xc] = val;
  }
}

__device__ __forceinline__ void store_out(float* __restrict__ base0, int64_t pitch, int y, int ny,
                                          int x, int nx, u64 v) {
  store_cols(base0 + (int64_t)y * pitch, x, nx, v);
  if (y == 1 || y == 2) store_cols(base0 - (int64_t)y * pitch, x, nx, v);
  if ((y == ny - 2 || y == ny - 3) && y >= 0)
    store_cols(base0 + (int64_t)(2 * (ny - 1) - y) * pitch, x, nx, v);
}

// One warp task: the band of kTY output rows starting at y0, columns of
// warp column bx.
template <bool kCoherent, bool kHint>
__device__ __forceinline__ u64 ld_row(const float* p, u64 pol) {
  // coherent (L2) loads when the planes were written earlier in the same launch;
  // with kHint the load carries the L2 eviction policy `pol`
  if constexpr (kHint) {
    u64 v;
    if constexpr (kCoherent)
      asm volatile("ld.global.cg.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    else
      asm volatile("ld.global.nc.L2::cache_hint.b64 %0, [%1], %2;" : "=l"(v) : "l"(p), "l"(pol));
    return v;
  } else {
    return kCoherent ? __ldcg(reinterpret_cast<const u64*>(p))
                     : __ldg(reinterpret_cast<const u64*>(p));
  }
}

template <bool kHint>
__device__ __forceinline__ void st_row(float* p, u64 v, u64 pol) {
  if constexpr (kHint)
    asm volatile("st.global.L2::cache_hint.b64 [%0], %1, %2;" ::"l"(p), "l"(v), "l"(pol) : "memory");
  else
    *reinterpret_cast<u64*>(p) = v;
}

// L2 eviction policy of an ensemble instance's plane accesses
__device__ __forceinline__ u64 l2_policy(int l2) {
  u64 p;
  if (l2 == kL2Stream)
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  else if (l2 == kL2StreamHalf)
    asm volatile("createpolicy.fractional.L2::evict_first.L2::evict_unchanged.b64 %0, 0.5;"
                 : "=l"(p));
  else
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}

template <bool kCH, bool kIso, int kTY, bool kCoherent = false, bool kHint = false>
__device__ __forceinline__ void sweep_task(const Explicit2DArgs& a, const float* in, float* out,
                                           const Coef& K, int bx, int y0, u64 pol = 0) {
  constexpr int kLag = kCH ? 2 : 1;
  constexpr int kWarm = 2 * kLag;  // rows consumed before the first finished row
  const int lane = threadIdx.x & 31;
  const int nx = a.nx, ny = a.ny;
  const int64_t pitch = a.pitch;
  const int x = bx * kOutCols - kPair + kPair * lane;  // real column of lo
  const bool writer = lane >= 1 && lane <= 30 && x < nx;
  // plain vector store unless this lane / band also owns mirror-frame cells
  const bool ghost_cols = x <= 2 || x + 1 >= nx - 3;
  const bool ghost_rows = y0 <= 2 || y0 + kTY + 3 >= ny;
  const bool plain = writer && !ghost_cols && !ghost_rows;
  // origin of the real mesh inside the ghost-padded planes
  const float* __restrict__ in0 = in + kGhost * pitch + kGhost;
  float* __restrict__ out0 = out + kGhost * pitch + kGhost;
  const float* src = in0 + (int64_t)(y0 - kLag) * pitch + x;
  Window w;
  u64 ahead[kAhead];  // rows k .. k+kAhead-1 in flight
#pragma unroll
  for (int j = 0; j < kAhead; ++j) {
    ahead[j] = ld_row<kCoherent, kHint>(src, pol);
    src += pitch;
  }
#pragma unroll
  for (int it = 0; it < kWarm; ++it) {  // fill the window, nothing to store yet
    const u64 P = ahead[0];
#pragma unroll
    for (int j = 0; j + 1 < kAhead; ++j) ahead[j] = ahead[j + 1];
    ahead[kAhead - 1] = ld_row<kCoherent, kHint>(src, pol);
    src += pitch;
    sweep_row<kCH, kIso>(P, w, K);
  }
#pragma unroll 6
  for (int it = 0; it < kTY; ++it) {
    const u64 P = ahead[0];
#pragma unroll
    for (int j = 0; j + 1 < kAhead; ++j) ahead[j] = ahead[j + 1];
    ahead[kAhead - 1] = ld_row<kCoherent, kHint>(src, pol);
    src += pitch;
    const u64 o = sweep_row<kCH, kIso>(P, w, K);
    const int y = y0 + it;
    if (plain)
      st_row<kHint>(out0 + (int64_t)y * pitch + x, o, pol);
    else if (writer && y < ny)
      store_out(out0, pitch, y, ny, x, nx, o);
  }
}

// One warp per block and one (column, band) task per warp: many small blocks
// spread evenly over the SMs and keep each scheduler fed from several warps.
template <bool kCH, bool kIso, int kTY>
__global__ void __launch_bounds__(kWarps * 32, PF_MINB) k_explicit2d(const Explicit2DArgs a) {
#if PF_PDL
  asm volatile("griddepcontrol.wait;" ::: "memory");  // the previous step is complete
#endif
  const int warp = threadIdx.x >> 5;
  const int y0 = (block_row() * kWarps + warp) * kTY;
  if (y0 < a.ny) sweep_task<kCH, kIso, kTY>(a, a.in, a.out, Coef{a.pair}, blockIdx.x, y0);
#if PF_PDL
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
#endif
}

// ---------------------------------------------------------------------------
// Batched ensembles of independent 2-D Allen-Cahn instances (different sizes
// and parameters).  Every instance has its own ghost-padded planes A/B and its
// own packed coefficients; the warp tasks of all instances -- (instance,
// column of 60, band of ty rows) -- form one list, so one launch advances the
// whole ensemble.  The persistent form keeps one launch resident for all
// steps, with a bounded grid barrier between steps.

template <bool kIso, bool kCoherent>
__device__ __forceinline__ void ensemble_task(const EnsTask& t, const Explicit2DArgs* inst,
                                              int parity) {
  const Explicit2DArgs& a = inst[t.inst];
#if PF_ENS_COEF == 0
  unsigned long long pair[19];
#pragma unroll
  for (int i = 0; i < 19; ++i) pair[i] = a.pair[i];
  const Coef K{pair};
#elif PF_ENS_COEF == 1
  const Coef K{a.pair};  // read through the instance table (L1-resident, warp-uniform)
#else
  __shared__ unsigned long long s_pair[kEnsThreads / 32][20];
  unsigned long long* sp = s_pair[threadIdx.x >> 5];
  __syncwarp();
  if ((threadIdx.x & 31) < 19) sp[threadIdx.x & 31] = a.pair[threadIdx.x & 31];
  __syncwarp();
  const Coef K{sp};
#endif
  const float* in = parity ? a.out : a.in;
  float* out = parity ? const_cast<float*>(a.in) : a.out;
  const u64 pol = l2_policy(a.l2);
  switch (t.ty) {
    case 6: sweep_task<false, kIso, 6, kCoherent, true>(a, in, out, K, t.bx, t.y0, pol); break;
    case 12: sweep_task<false, kIso, 12, kCoherent, true>(a, in, out, K, t.bx, t.y0, pol); break;
    default: sweep_task<false, kIso, 24, kCoherent, true>(a, in, out, K, t.bx, t.y0, pol); break;
  }
}

template <bool kIso>
__global__ void __launch_bounds__(kEnsThreads, PF_ENS_MINB) k_ensemble_step(const EnsTask* __restrict__ tasks,
                                                              int ntasks,
                                                              const Explicit2DArgs* inst,
                                                              int parity) {
  const int warps = kEnsThreads / 32;
  for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < ntasks; t += gridDim.x * warps)
    ensemble_task<kIso, false>(tasks[t], inst, parity);
}

// Grid-wide barrier for a co-resident (cooperative) grid.  bar[0] counts
// arrivals, bar[1] is the generation, bar[2] the error flag.  A block that
// waits longer than `limit` clock cycles sets the flag and reports failure.
__device__ bool grid_barrier(unsigned* bar, long long limit) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x - 1) {
      bar[0] = 0;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > limit) {
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ok != 0;
}

template <bool kIso>
__global__ void __launch_bounds__(kEnsThreads, PF_ENS_MINB) k_ensemble_persistent(
    const EnsTask* __restrict__ tasks, int ntasks, const Explicit2DArgs* inst, int n_steps,
    unsigned* bar, long long limit) {
  const int warps = kEnsThreads / 32;
  for (int s = 0; s < n_steps; ++s) {
    for (int t = blockIdx.x * warps + (threadIdx.x >> 5); t < ntasks; t += gridDim.x * warps)
      ensemble_task<kIso, true>(tasks[t], inst, s & 1);
    if (!grid_barrier(bar, limit)) return;
  }
}

// Self-test of the bounded barrier: `extra` phantom arrivals are expected that
// never come, so every block's wait must expire and set the error flag.
__global__ void k_barrier_selftest(unsigned* bar, long long limit, int extra) {
  __shared__ int ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    ok = 1;
    volatile unsigned* vgen = bar + 1;
    const unsigned gen = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(bar, 1u);
    if (arrived == gridDim.x + extra - 1) {
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == gen) {
        if (clock64() - t0 > limit) {
          atomicExch(bar + 2, 1u);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
  }
  __syncthreads();
}

// all instances' plain states (packed) <-> their padded working planes
// (grid.y strides over the instances, so any count fits in one launch; blocks
// stride over rows and threads over columns, so no index is divided)
__global__ void k_ens_to_work(const float* __restrict__ packed, const int64_t* __restrict__ off,
                              const Explicit2DArgs* inst, int count, float sub) {
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const Explicit2DArgs& a = inst[k];
    const int nx = a.nx, ny = a.ny;
    const int64_t pitch = a.pitch;
    const float* in = packed + off[k];
    for (int v = blockIdx.x; v < a.rows; v += gridDim.x) {
      const int y = v - kGhost;
      const bool row = y >= -kGhost && y < ny + kGhost;
      const int64_t src = (int64_t)reflect_row(y, ny) * nx;
      float* dA = const_cast<float*>(a.in) + v * pitch;
      float* dB = a.out + v * pitch;
      for (int u = threadIdx.x; u < pitch; u += blockDim.x) {
        const int x = u - kGhost;
        float val = 0.0f;
        if (row && x >= -kGhost && x < nx + kGhost) val = in[src + reflect_col(x, nx)] - sub;
        dA[u] = val;
        dB[u] = val;
      }
    }
  }
}

__global__ void k_ens_from_work(float* __restrict__ packed, const int64_t* __restrict__ off,
                                const Explicit2DArgs* inst, int count, int parity, float add) {
  for (int k = blockIdx.y; k < count; k += gridDim.y) {
    const Explicit2DArgs& a = inst[k];
    const int nx = a.nx;
    const float* work = parity ? a.out : a.in;
    float* out = packed + off[k];
    for (int y = blockIdx.x; y < a.ny; y += gridDim.x) {
      const float* src = work + (int64_t)(y + kGhost) * a.pitch + kGhost;
      float* dst = out + (int64_t)y * nx;
      for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = src[x] + add;
    }
  }
}

// Plain <-> padded working layout.  Working cell (u, v) holds real node
// (reflect(u - kGhost), reflect(v - kGhost)) minus/plus the shift; padding
// beyond the ghost frame is zero.  Blocks stride over rows, threads over
// columns.
__global__ void k_to_work(const float* __restrict__ in, float* __restrict__ work, int nx, int ny,
                          int64_t pitch, int rows, float sub) {
  for (int v = blockIdx.x; v < rows; v += gridDim.x) {
    const int y = v - kGhost;
    const bool row = y >= -kGhost && y < ny + kGhost;
    const int64_t src = (int64_t)reflect_row(y, ny) * nx;
    float* dst = work + v * pitch;
    for (int u = threadIdx.x; u < pitch; u += blockDim.x) {
      const int x = u - kGhost;
      float val = 0.0f;
      if (row && x >= -kGhost && x < nx + kGhost) val = in[src + reflect_col(x, nx)] - sub;
      dst[u] = val;
    }
  }
}

__global__ void k_from_work(const float* __restrict__ work, float* __restrict__ out, int nx,
                            int ny, int64_t pitch, float add) {
  for (int y = blockIdx.x; y < ny; y += gridDim.x) {
    const float* src = work + (int64_t)(y + kGhost) * pitch + kGhost;
    float* dst = out + (int64_t)y * nx;
    for (int x = threadIdx.x; x < nx; x += blockDim.x) dst[x] = src[x] + add;
  }
}

#ifndef PF_TY_CH
#define PF_TY_CH 6
#endif
#ifndef PF_TY_AC
#define PF_TY_AC 12
#endif
constexpr int kTYAc = PF_TY_AC;  // output rows per warp band (a multiple of the unroll of 6)
constexpr int kTYCh = PF_TY_CH;

template <bool kCH, bool kIso, int kTY>
cudaError_t launch(const Explicit2DArgs& a, cudaStream_t s) {
  const dim3 grid = row_grid((a.nx + kOutCols - 1) / kOutCols, (a.ny + kWarps * kTY - 1) / (kWarps * kTY));
#if PF_PDL
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = dim3(kWarps * 32);
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_explicit2d<kCH, kIso, kTY>, a);
#else
  k_explicit2d<kCH, kIso, kTY><<<grid, kWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
#endif
}

bool is_iso(const Stencil2D& k) { return k.cx == k.cd && k.cy == k.cd; }

}  // namespace

cudaError_t launch_ac2d(const Explicit2DArgs& a, cudaStream_t s) {
  return is_iso(a.k1) ? launch<false, true, kTYAc>(a, s) : launch<false, false, kTYAc>(a, s);
}

cudaError_t launch_ch2d(const Explicit2DArgs& a, cudaStream_t s) {
  return (is_iso(a.k1) && is_iso(a.k2)) ? launch<true, true, kTYCh>(a, s)
                                        : launch<true, false, kTYCh>(a, s);
}

void pack_explicit2d(Explicit2DArgs& a) {
  auto pk_host = [](float v) {
    unsigned int b;
    memcpy(&b, &v, 4);
    return (unsigned long long)b | ((unsigned long long)b << 32);
  };
  a.pair[0] = pk_host(kGLo);
  a.pair[1] = pk_host(kGHi);
  a.pair[2] = pk_host(-kGLo);
  a.pair[3] = pk_host(a.p0);
  a.pair[4] = pk_host(a.p1);
  a.pair[5] = pk_host(a.p2);
  a.pair[6] = pk_host(a.p3);
  const Stencil2D* st[2] = {&a.k1, &a.k2};
  for (int s = 0; s < 2; ++s) {
    a.pair[7 + 6 * s + 0] = pk_host(st[s]->c0 - st[s]->cd);
    a.pair[7 + 6 * s + 1] = pk_host(st[s]->cd);
    a.pair[7 + 6 * s + 2] = pk_host(st[s]->c0);
    a.pair[7 + 6 * s + 3] = pk_host(st[s]->cx);
    a.pair[7 + 6 * s + 4] = pk_host(st[s]->cy);
    a.pair[7 + 6 * s + 5] = pk_host(st[s]->cd);
  }
}

cudaError_t launch_ensemble_step(const EnsTask* tasks, int ntasks, const Explicit2DArgs* inst,
                                 int parity, bool iso, int grid, cudaStream_t s) {
  if (iso)
    k_ensemble_step<true><<<grid, kEnsThreads, 0, s>>>(tasks, ntasks, inst, parity);
  else
    k_ensemble_step<false><<<grid, kEnsThreads, 0, s>>>(tasks, ntasks, inst, parity);
  return cudaGetLastError();
}

int ensemble_persistent_grid(bool iso) {
  int dev = 0, sms = 0, per = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  cudaError_t e = iso ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per, k_ensemble_persistent<true>, kEnsThreads, 0)
                      : cudaOccupancyMaxActiveBlocksPerMultiprocessor(
                            &per, k_ensemble_persistent<false>, kEnsThreads, 0);
  if (e != cudaSuccess) return 0;
  return sms * per;
}

cudaError_t launch_ensemble_persistent(const EnsTask* tasks, int ntasks, const Explicit2DArgs* inst,
                                       int n_steps, unsigned* bar, long long limit, bool iso,
                                       int grid, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(kEnsThreads);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return iso ? cudaLaunchKernelEx(&cfg, k_ensemble_persistent<true>, tasks, ntasks, inst, n_steps,
                                  bar, limit)
             : cudaLaunchKernelEx(&cfg, k_ensemble_persistent<false>, tasks, ntasks, inst, n_steps,
                                  bar, limit);
}

cudaError_t launch_ens_to_work(const float* packed, const int64_t* off, const Explicit2DArgs* inst,
                               int count, float shift, cudaStream_t s) {
  const unsigned gy = count < (int)kMaxGridY ? (unsigned)count : kMaxGridY;
  k_ens_to_work<<<dim3(64, gy), 256, 0, s>>>(packed, off, inst, count, shift);
  return cudaGetLastError();
}

cudaError_t launch_ens_from_work(float* packed, const int64_t* off, const Explicit2DArgs* inst,
                                 int count, int parity, float shift, cudaStream_t s) {
  const unsigned gy = count < (int)kMaxGridY ? (unsigned)count : kMaxGridY;
  k_ens_from_work<<<dim3(64, gy), 256, 0, s>>>(packed, off, inst, count, parity, shift);
  return cudaGetLastError();
}

cudaError_t launch_barrier_selftest(unsigned* bar, long long limit, int extra, cudaStream_t s) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_barrier_selftest, bar, limit, extra);
}

int work_pitch(int nx) {
  const int gx = (nx + kOutCols - 1) / kOutCols;
  const int p = gx * kOutCols + 2 * kGhost + 2 * kPair;
  return (p + 3) / 4 * 4;
}

int work_rows(int ny) {
  // the last band reads up to ty + kLag + kAhead rows past its first row
  int ty = kTYAc > kTYCh ? kTYAc : kTYCh;
  if (ty < kMaxEnsTY) ty = kMaxEnsTY;
  return ny + ty + kAhead + 2 * kGhost + 4;
}

cudaError_t launch_to_work(const float* in, float* work, int nx, int ny, float shift,
                           cudaStream_t s) {
  int64_t blocks = work_rows(ny);
  if (blocks > 16 * (int64_t)device_sm_count()) blocks = 16 * (int64_t)device_sm_count();
  k_to_work<<<(unsigned)blocks, 256, 0, s>>>(in, work, nx, ny, work_pitch(nx), work_rows(ny),
                                             shift);
  return cudaGetLastError();
}

cudaError_t launch_from_work(const float* work, float* out, int nx, int ny, float shift,
                             cudaStream_t s) {
  int64_t blocks = ny;
  if (blocks > 16 * (int64_t)device_sm_count()) blocks = 16 * (int64_t)device_sm_count();
  k_from_work<<<(unsigned)blocks, 256, 0, s>>>(work, out, nx, ny, work_pitch(nx), shift);
  return cudaGetLastError();
}

}  // namespace pf
