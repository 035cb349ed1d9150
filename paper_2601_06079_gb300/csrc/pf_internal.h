// Internal declarations shared by the libpf translation units (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <string>

#include "../../include/pf.h"

namespace pf {

// Gauss points of the 2-point rule on the unit interval, (1 -+ 1/sqrt 3)/2.
// g_lo = N_0 at the upper point = N_1 at the lower point, and vice versa.
constexpr float kGHi = 0.78867513459481288225f;
constexpr float kGLo = 0.21132486540518711775f;

// 2-D launches put rows of blocks on grid.y, which holds at most 65,535; a
// taller mesh (up to 2^20 node rows) continues on grid.z.  block_row() is the
// block's row; rows past the last (when `rows` is not a multiple of the y
// extent) must return at once.
constexpr unsigned kMaxGridY = 65535;
inline dim3 row_grid(unsigned cols, unsigned rows) {
  const unsigned y = rows == 0 ? 1 : (rows < kMaxGridY ? rows : kMaxGridY);
  return dim3(cols, y, (rows + y - 1) / y);
}
#ifdef __CUDACC__
__device__ __forceinline__ int block_row() { return (int)(blockIdx.z * gridDim.y + blockIdx.y); }
#endif

// Raises a kernel's dynamic shared-memory limit to `bytes` on the current
// device.  The attribute belongs to the device, so `done` (one per kernel
// instantiation) records the devices 0..63 already raised; others are set on
// every call.  Safe to call from several host threads.
template <class K>
inline cudaError_t raise_smem_limit(K* kernel, int bytes, std::atomic<unsigned long long>& done) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = dev >= 0 && dev < 64 ? 1ull << dev : 0ull;
  if (bit && (done.load(std::memory_order_acquire) & bit)) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess && bit) done.fetch_or(bit, std::memory_order_acq_rel);
  return e;
}

// Streaming multiprocessors of the current device (cached per device 0..63).
// Grid sizes that must not change between calls on one device (fixed-order
// reductions, workspace sizes) derive from it, never from a constant.
inline int device_sm_count() {
  static std::atomic<int> cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev >= 0 && dev < 64) {
    const int c = cache[dev].load(std::memory_order_relaxed);
    if (c > 0) return c;
  }
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    sms = 1;
  if (dev >= 0 && dev < 64) cache[dev].store(sms, std::memory_order_relaxed);
  return sms;
}

// Assembled 9-point Q1 stiffness stencil on a uniform 2-D grid, pre-scaled:
// (K v)_i = c0 v_i + cx (v_W + v_E) + cy (v_S + v_N) + cd (v_SW + v_SE + v_NW + v_NE).
struct Stencil2D {
  float c0, cx, cy, cd;
};

// Arguments of one fused explicit step on a 2-D mesh.  The state is the
// shifted FP32 variable d = u - shift; the mirror extension about boundary
// nodes reproduces the zero-flux Q1 operators divided by the lumped mass, so
// every node uses the interior stencil and the interior mass.
struct Explicit2DArgs {
  const float* in;
  float* out;
  int nx, ny;
  int rows;       // rows of the ghost-padded working planes
  int64_t pitch;  // row pitch of the ghost-padded working planes (floats)
  // f'(shift + d) / 4 as p0 + d (p1 + d (p2 + d p3)), times the stage factor
  float p0, p1, p2, p3;
  Stencil2D k1;  // AC: -dt L kappa / m * K;   CH: kappa / m * K  (mu stage)
  Stencil2D k2;  // CH: -dt M / m * K          (c stage)
  // the same constants duplicated into FP32 pairs for the packed f32x2 path
  // (filled by pack_explicit2d): g_lo, g_hi, -g_lo, p0..p3, then per stencil
  // a = c0 - cd, b = cd, c0, cx, cy, cd
  unsigned long long pair[7 + 12];
  // L2 eviction priority of the working planes' row loads and stores in the
  // ensemble sweep (kL2Normal, kL2Stream, kL2StreamHalf); single-mesh steps
  // ignore it
  int l2;
};
void pack_explicit2d(Explicit2DArgs& a);
constexpr int kL2Normal = 0;      // evict_normal
constexpr int kL2Stream = 1;      // evict_first: the lines go first when L2 needs room
constexpr int kL2StreamHalf = 2;  // evict_first for half of the lines, the rest unchanged

cudaError_t launch_ac2d(const Explicit2DArgs& a, cudaStream_t s);

// Coupled Allen-Cahn / Cahn-Hilliard step (planes [c - shift; eta], no frame).
struct Coupled2DArgs {
  const float* in;
  float* out;
  int nx, ny;
  float fa[5], dfa[4], fb[3], dfb[2];  // f_alpha, f_beta and derivatives in d = c - shift
  float h[6], dh[5];                   // h(eta), h'(eta)
  Stencil2D k1;                        // kappa_eta / m K
  Stencil2D k2;                        // -dt M_c / m K
  float neg_dt_meta;                   // -dt M_eta
};
cudaError_t launch_coupled2d(const Coupled2DArgs& a, cudaStream_t s);
// The plain two-pass comparison form (d, mu, out: nx x ny arrays without frame).
cudaError_t launch_plain2d(bool ch, const Explicit2DArgs& a, const float* d, float* mu, float* out,
                           cudaStream_t s);

// Batched ensembles of 2-D Allen-Cahn instances.
struct EnsTask {
  int inst;  // instance
  int bx;    // warp column (60 output columns each)
  int y0;    // first output row of the band
  int ty;    // band height: 6, 12 or 24
};
constexpr int kEnsThreads = 128;
constexpr int kMaxEnsTY = 24;
constexpr int kEnsOutCols = 60;
cudaError_t launch_ensemble_step(const EnsTask* tasks, int ntasks, const Explicit2DArgs* inst,
                                 int parity, bool iso, int grid, cudaStream_t s);
int ensemble_persistent_grid(bool iso);
cudaError_t launch_barrier_selftest(unsigned* bar, long long limit, int extra, cudaStream_t s);
cudaError_t launch_ensemble_persistent(const EnsTask* tasks, int ntasks, const Explicit2DArgs* inst,
                                       int n_steps, unsigned* bar, long long limit, bool iso,
                                       int grid, cudaStream_t s);
cudaError_t launch_ens_to_work(const float* packed, const int64_t* off, const Explicit2DArgs* inst,
                               int count, float shift, cudaStream_t s);
cudaError_t launch_ens_from_work(float* packed, const int64_t* off, const Explicit2DArgs* inst,
                                 int count, int parity, float shift, cudaStream_t s);
cudaError_t launch_ch2d(const Explicit2DArgs& a, cudaStream_t s);
// Ghost-padded working planes: work_pitch(nx) x work_rows(ny) floats each.
int work_pitch(int nx);
int work_rows(int ny);
cudaError_t launch_to_work(const float* in, float* work, int nx, int ny, float shift,
                           cudaStream_t s);
cudaError_t launch_from_work(const float* work, float* out, int nx, int ny, float shift,
                             cudaStream_t s);

// Energy / mass diagnostics (Eq. 5-6), FP64 accumulation, deterministic.
struct Energy2DArgs {
  const float* d;  // shifted state (one field)
  int nx, ny;
  double hx, hy;
  float shift;
  float q0, q1, q2, q3, q4;  // f(shift + d) = q0 + d (q1 + d (q2 + d (q3 + d q4)))
  float kappa;
};
int energy2d_blocks(int nx, int ny);
cudaError_t launch_energy2d(const Energy2DArgs& a, double* partials, double* result,
                            cudaStream_t s);

// 2-D Cahn-Hilliard with a per-node mobility field: explicit step and its
// discrete adjoint (plain row-major planes, shifted state d = c - s).
struct ChMobArgs {
  const float* d;       // shifted state at which the operators are evaluated
  const float* mfield;  // mobility multiplier per node
  int nx, ny;
  float p0, p1, p2, p3;  // f'(s + d) = p0 + d (p1 + d (p2 + d p3))
  float s0, s1, s2;      // f''(s + d) = s0 + d (s1 + d s2)
  Stencil2D k;           // Q1 stiffness stencil / cell
  float kappa, M, W, dt, ihx, ihy;
  double cell;
  float ngm;  // -dt M cell, the factor of the mobility gradient (reverse step)
};
int ch_mob_blocks(int nx, int ny);
cudaError_t launch_ch_mob_step(const ChMobArgs& a, float* out, cudaStream_t s);
// grad_hi / grad_lo: the running mobility gradient as a compensated FP32 pair
// per node (both null: not accumulated); grad_to_double writes hi + lo in FP64.
cudaError_t launch_ch_adj_step(const ChMobArgs& a, const float* yin, float* yout,
                               float* grad_hi, float* grad_lo, double* acc, cudaStream_t s);
cudaError_t launch_grad_to_double(const float* hi, const float* lo, double* out, int64_t n,
                                  cudaStream_t s);
cudaError_t launch_loss(const float* d, float shift, const float* target, int nx, int ny,
                        double cell, int nodal, float* y, double* partials, double* out,
                        cudaStream_t s);
cudaError_t launch_colsum(const double* in, int nb, int stride, int k, double* out,
                          cudaStream_t s);
cudaError_t launch_mass_scale(const float* y, int nx, int ny, double cell, float* out,
                              cudaStream_t s);
cudaError_t launch_add(const float* in, float* out, int64_t n, float add, cudaStream_t s);

// 3-D implicit operators (Eq. 13-14), scaled by the lumped mass unless unscaled.
struct Implicit3DArgs {
  const float* U;  // state at which r / H is evaluated (nf planes)
  const float* W;  // JVP: direction v; residual: U^n
  float* out;      // nf planes
  int nx, ny, nz, nf;
  int double_well;  // 1: f = W u^2 (1-u)^2 (nf == 1); 0: Fan-Chen
  float dw2;        // 2 W
  float alpha, two_gamma, four_gamma, cb2g, c3b6g;  // Fan-Chen: a, 2g, 4g, b - 2g, 3b - 6g
  float kg[3];      // 2 kappa / h_d^2: weights of the element gradient term per axis
  float inv_dt, mob;
  float cell;       // hx hy hz
  int unscaled;     // multiply the result by the lumped mass m_i
};
cudaError_t launch_residual3d(const Implicit3DArgs& a, cudaStream_t s);

// The same operators on a 2-D mesh with the double well: Allen-Cahn (one
// plane) or the split Cahn-Hilliard system (planes [c; mu]).
struct Implicit2DArgs {
  const float* U;  // state at which r / H is evaluated (CH: [c; mu])
  const float* W;  // JVP: direction v; residual: U^n (CH: c^n in the first plane)
  float* out;
  int nx, ny;
  float dw2;       // 2 W
  Stencil2D k;     // kappa / m K
  Stencil2D km;    // CH: M_c / m K
  float inv_dt, mob;
  float cell;      // hx hy
  int unscaled;    // multiply the result by the lumped mass m_i
  int ch;          // 1: split Cahn-Hilliard
};
cudaError_t launch_residual2d(const Implicit2DArgs& a, cudaStream_t s);
cudaError_t launch_jvp2d(const Implicit2DArgs& a, cudaStream_t s);
cudaError_t launch_jvp3d(const Implicit3DArgs& a, cudaStream_t s);

// Eshelby-inclusion elasticity (Eq. 3-4, III.1): K u with the element
// stiffness ke[(a*3+i)*24 + b*3+j] of the uniform box element and its
// assembled interior stencil ks[(o*3+i)*3+j], o = (dz+1)*9 + (dy+1)*3 + (dx+1).
struct Elastic3DArgs {
  const float* u;
  float* out;
  double* dot;  // optional: per-block FP64 partials of u . out (elastic_apply_blocks entries)
  int nx, ny, nz;
  int constrain;  // zero the rows of the symmetry-plane constraints
  float ke[24 * 24];
  float ks[27 * 9];
};
// load: w d_i N_a(q) s(q) summed per node; s = scale * phi(|x_q|) (unit = 0,
// phi = (1 - tanh(l (r - a))) / 2) or scale (unit = 1)
struct ElasticLoadArgs {
  int nx, ny, nz;
  int unit, constrain;
  float hx, hy, hz, ihx, ihy, ihz, wq, scale, l, a;
};
int elastic_apply_blocks(int nx, int ny, int nz);
int cg_blocks();  // blocks (and r.r partials) of launch_cg_xr
cudaError_t launch_elastic_apply(const Elastic3DArgs& a, cudaStream_t s);
cudaError_t launch_sum_part(const double* part, int nb, double* out, cudaStream_t s);
cudaError_t launch_elastic_load(const ElasticLoadArgs& a, float* f, cudaStream_t s);
cudaError_t launch_elastic_constrain(float* v, int nx, int ny, int nz, cudaStream_t s);
// CG updates with device scalars sc[0..1] = r.r (ping-pong by slot), sc[2] = p.Ap;
// launch_cg_xr also leaves the new r.r as cg_blocks() FP64 partials in part
cudaError_t launch_cg_xr(float* x, float* r, const float* p, const float* Ap, int64_t n,
                         const double* sc, int slot, double* part, cudaStream_t s);
cudaError_t launch_cg_p(const float* r, float* p, int64_t n, const double* sc, int slot,
                        cudaStream_t s);

// Krylov vector kernels (FP32 vectors, FP64 inner products).
constexpr int kMaxBasis = 32;  // GMRES restart length + 1
struct LinComb {
  float c[kMaxBasis];
};
int krylov_partial_blocks();
// The reductions below finish in the same launch: the last block sums the
// per-block partials (krylov_partial_blocks() x k doubles) in a fixed order.
// count: a device counter that is 0 between calls (each call leaves it 0).
cudaError_t launch_dots(const float* V, int64_t ldv, int k, const float* w, int64_t n,
                        double* partials, double* out, unsigned* count, cudaStream_t s);
cudaError_t launch_update(const float* V, int64_t ldv, int k, const double* coef, float* w,
                          int64_t n, double* partials, double* norm_out, unsigned* count,
                          cudaStream_t s);
// w <- w - sum_j coef[j] V_j, then out[j] = V_j . w (j < k) for the updated w,
// in one pass (results identical to launch_update followed by launch_dots)
cudaError_t launch_update_dots(const float* V, int64_t ldv, int k, const double* coef, float* w,
                               int64_t n, double* partials, double* out, unsigned* count,
                               cudaStream_t s);
cudaError_t launch_axpby(float a, const float* x, float b, float* y, int64_t n, cudaStream_t s);
cudaError_t launch_mass_mul(const float* in, float* out, int nx, int ny, int nz, int nf,
                            double cell, float a, int inverse, cudaStream_t s);
cudaError_t launch_lincomb(const float* V, int64_t ldv, int k, const LinComb& y, float* x,
                           int64_t n, cudaStream_t s);
cudaError_t launch_mass_norm(const float* g, int nx, int ny, int nz, int nf, double cell,
                             double* partials, double* out, unsigned* count, cudaStream_t s);

// Learned surrogate: 3x3x3 convolution kernels (BF16 tensor cores) and the
// element-wise layers around them.  Activations NDHWC BF16.
// mma.sync implicit GEMM (any D even, H and W multiples of 8):
cudaError_t launch_conv3d(int cin, int cout, const void* x, const void* wt, const float* bias,
                          int relu, void* y16, float* y32, int B, int D, int H, int W, int grid,
                          cudaStream_t s);
// tcgen05 + TMA implicit GEMM (D even, H multiple of 8, any W); *err is set
// to 1 when a pipeline wait expired (the output is then incomplete).
// selftest = 1 issues no input copies, so that the waits must expire.
bool conv3d_tc_shape_ok(int B, int D, int H, int W);
cudaError_t launch_conv3d_tc(int cin, int cout, const void* x, const void* wt, const float* bias,
                             int relu, void* y16, float* y32, int B, int D, int H, int W,
                             int* err, cudaStream_t s, int selftest = 0);
int conv_wgrad_blocks(int B, int D, int H, int W, int max_blocks);
// Weight gradient on tcgen05 (k_wgrad_tc.cu): needs H and W multiples of 8;
// part holds wgrad_tc_part_floats() floats of per-block partial sums; err is
// the pipeline-timeout flag.
bool wgrad_tc_shape_ok(int B, int D, int H, int W);
int wgrad_tc_blocks();
size_t wgrad_tc_part_floats();
cudaError_t launch_wgrad_tc(int cin, int cout, const void* x, const void* dy, float* part,
                            float* dw, int B, int D, int H, int W, int* err, cudaStream_t s);
cudaError_t launch_conv3d_wgrad(int cin, int cout, const void* x, const void* dy, float* part,
                                float* dw, int B, int D, int H, int W, int blocks, cudaStream_t s);
// db[c] = sum over voxels of dy[v][c]; scratch: >= bias_grad_blocks() * C floats
int bias_grad_blocks();
cudaError_t launch_bias_grad(const void* dy, int C, int64_t nvox, float* db, float* scratch,
                             cudaStream_t s);
cudaError_t launch_planar_to_ndhwc(const float* in, int nf, int C, int B, int64_t V, int mode,
                                   const float* sig, void* out, cudaStream_t s);
cudaError_t launch_ndhwc_to_planar_add(const float* y, int C, int nf, int B, int64_t V,
                                       const float* base, int nb, int mode, const float* sig,
                                       float* out, cudaStream_t s);
// sig[b]: the input unit (a * RMS of U^n - U^{n-1}; a for mode 0); sigo[b]:
// the output unit (= sig, except mode 2: a * RMS of U^n - 2 U^{n-1} + U^{n-2},
// floored at 1e-3 sig[b])
cudaError_t launch_incr_scale(const float* x, int nf, int B, int64_t V, float a, int mode,
                              double* part, int nblk, float* sig, float* sigo, cudaStream_t s);
cudaError_t launch_pool(const void* in, int B, int D, int H, int W, int C, void* out,
                        cudaStream_t s);
cudaError_t launch_up_add(const void* coarse, const void* skip, int B, int D, int H, int W, int C,
                          void* out, cudaStream_t s);
cudaError_t launch_down_sum(const void* g, int B, int D, int H, int W, int C, void* out,
                            cudaStream_t s);
cudaError_t launch_pool_back_add(const void* gc, int B, int D, int H, int W, int C, void* acc,
                                 cudaStream_t s);
cudaError_t launch_relu_mask(void* g, const void* y, int64_t n, cudaStream_t s);
cudaError_t launch_mse(const float* pred, int C, int nf, int nxc, int B, int D, int H, int W,
                       const float* x, const float* y, int mode, const float* sig, float c,
                       float scale, float* r, float* q, void* grad, double* partials,
                       double* loss, cudaStream_t s);
cudaError_t launch_convert_weights(const float* w, int ci, int co, void* fwd, void* bwd,
                                   cudaStream_t s);
// All layers' conversions in one launch: layer l converts w[l] (27 x co x ci
// FP32) into fwd[l] (and bwd[l] unless null), as launch_convert_weights does.
constexpr int kMaxConvertLayers = 16;
struct ConvertTable {
  const float* w[kMaxConvertLayers];
  void* fwd[kMaxConvertLayers];
  void* bwd[kMaxConvertLayers];
  int ci[kMaxConvertLayers], co[kMaxConvertLayers];
  int n;
};
cudaError_t launch_convert_weights_all(const ConvertTable& t, cudaStream_t s);
cudaError_t launch_adam(float* p, float* m, float* v, const float* g, int64_t n, float lr,
                        float b1, float b2, float eps, int step, cudaStream_t s);

}  // namespace pf
