// C ABI of libpf: context, workspace carving, parameter derivation and the
// host-side drivers that enqueue the kernels.  No device memory is allocated
// here; all scratch lives in the caller's workspace.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>
#include <string>

#include "pf_internal.h"

struct pf_ctx {
  int dim = 2;
  int64_t n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  pf_model model = PF_MODEL_AC;
  int nf = 1;
  cudaStream_t stream = nullptr;

  size_t ws_bytes = 0;     // workspace for every operation
  size_t ws_explicit = 0;  // prefix that explicit steps and diagnostics use
  size_t ws_bound = 0;     // bytes bound by pf_bind_workspace
  char* ws = nullptr;
  pf_params par{};
  bool par_set = false;
  int form = PF_FORM_FUSED_GRAPH;  // execution form of the 2-D explicit step
  pf::Coupled2DArgs cp{};          // coupled AC-CH step constants
  pf::Implicit2DArgs im2{};        // 2-D implicit operators (AC)

  // workspace segments
  float* buf_a = nullptr;
  float* buf_b = nullptr;
  double* partials = nullptr;
  double* result = nullptr;

  // derived coefficients
  pf::Explicit2DArgs ex{};
  pf::Implicit3DArgs im{};
  pf::ChMobArgs mob{};

  // 3-D workspace segments (each n_fields * N floats)
  float* u = nullptr;   // current iterate / state
  float* un = nullptr;  // U^n
  float* g = nullptr;   // scaled residual M^-1 R
  float* d = nullptr;   // Newton correction
  float* basis = nullptr;  // kMaxBasis Krylov vectors
  int64_t ldv = 0;         // floats between consecutive Krylov vectors
  double* small = nullptr; // h1[32], h2[32], scalars
  unsigned* count = nullptr;  // block counter of the single-launch reductions (0 between calls)
  bool count_zeroed = false;  // set once the counter has been cleared after a bind

  // CUDA graph of kGraphSteps explicit steps buf_a -> ... -> buf_a
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;
  // the same for the mobility-field steps, with the field it was captured with
  cudaGraphExec_t mob_graph = nullptr;
  const float* mob_graph_field = nullptr;

  // batched ensemble (count > 0): instances' sizes, tuned band heights, device arrays
  int ens_count = 0;
  std::vector<int64_t> ens_nx, ens_ny;
  std::vector<double> ens_hx, ens_hy;
  std::vector<int> ens_ty;
  std::vector<int64_t> ens_off;                 // packed-state offsets (count + 1)
  std::vector<pf::Explicit2DArgs> ens_args;     // host copy of the per-instance arguments
  std::vector<pf::EnsTask> ens_host_tasks;
  pf::Explicit2DArgs* ens_dargs = nullptr;
  pf::EnsTask* ens_tasks = nullptr;
  int64_t* ens_doff = nullptr;
  unsigned* ens_bar = nullptr;
  int ens_ntasks = 0;
  bool ens_iso = true;

  std::string err;
};

namespace {

constexpr int kGraphSteps = 64;  // even, so a replay returns to buf_a

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

int64_t nnodes(const pf_ctx* c) { return c->n[0] * c->n[1] * (c->dim == 3 ? c->n[2] : 1); }

pf_status fail(pf_ctx* c, pf_status s, const char* fmt, ...) {
  if (c) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->err = buf;
  }
  return s;
}

pf_status cuda_fail(pf_ctx* c, cudaError_t e, const char* where) {
  return fail(c, PF_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define PF_CUDA(call)                                      \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

// Workspace layout.  Everything explicit steps and the diagnostics touch
// comes first (`explicit_total` bytes): the 2-D working planes, the reduction
// buffers and, in 3-D, the residual vector G.  The implicit step's vectors
// (U, U^n, the Newton correction and the Krylov basis) follow, so a mesh that
// is only stepped explicitly binds the prefix alone.
struct Layout {
  size_t a, b, partials, result, vec, vecs, small, explicit_total, total;
};

constexpr int kVec3d = 4;  // U, U^n, G, D before the Krylov basis
constexpr double kNoOversolve = 0.1;  // GMRES floor, as a fraction of Newton's tolerance

// meshes with the implicit step (and its Krylov vectors): 3-D, and 2-D Allen-Cahn
bool has_implicit(const pf_ctx* c) {
  return c->ens_count == 0 &&
         (c->dim == 3 || c->model == PF_MODEL_AC || c->model == PF_MODEL_CH);
}

// 2-D Cahn-Hilliard solves the split system for [c; mu]: two planes per vector
bool split_ch(const pf_ctx* c) { return c->dim == 2 && c->model == PF_MODEL_CH; }
int imp_nf(const pf_ctx* c) { return split_ch(c) ? 2 : c->nf; }

Layout layout(const pf_ctx* c) {
  Layout L{};
  size_t off = 0;
  if (c->dim == 2) {
    const size_t field = align_up(sizeof(float) * (size_t)pf::work_pitch((int)c->n[0]) *
                                      pf::work_rows((int)c->n[1]) * c->nf,
                                  256);
    L.a = off;
    off += field;
    L.b = off;
    off += field;
  }
  L.partials = off;
  const size_t np = (size_t)std::max(2 * 1024, pf::krylov_partial_blocks() * pf::kMaxBasis);
  off += align_up(sizeof(double) * np, 256);
  L.result = off;
  off += 256;
  L.small = off;
  off += align_up(sizeof(double) * 4 * pf::kMaxBasis, 256);
  L.explicit_total = off;
  if (has_implicit(c)) {
    L.vec = align_up(sizeof(float) * (size_t)nnodes(c) * imp_nf(c), 256);
    L.vecs = off;  // G first: the 3-D explicit step needs it
    if (c->dim == 3) L.explicit_total = off + L.vec;
    off += L.vec * (kVec3d + pf::kMaxBasis);
  }
  L.total = off;
  return L;
}

// true once the bound workspace covers the implicit step's vectors
bool implicit_bound(const pf_ctx* c) { return c->ws && c->ws_bound >= c->ws_bytes; }

pf_status need_implicit_ws(pf_ctx* c) {
  if (implicit_bound(c)) return PF_OK;
  return fail(c, PF_ERR_STATE,
              "the bound workspace (%zu bytes) covers explicit steps only; implicit steps "
              "need %zu bytes",
              c->ws_bound, c->ws_bytes);
}

// 9-point Q1 stiffness stencil for spacing hx, hy (2x2 Gauss is exact for it).
pf::Stencil2D stiffness2d(double hx, double hy, double scale) {
  const double rx = hy / hx, ry = hx / hy;
  pf::Stencil2D s;
  s.c0 = (float)(scale * (4.0 / 3.0) * (rx + ry));
  s.cx = (float)(scale * (-(2.0 / 3.0) * rx + (1.0 / 3.0) * ry));
  s.cy = (float)(scale * ((1.0 / 3.0) * rx - (2.0 / 3.0) * ry));
  s.cd = (float)(scale * (-(1.0 / 6.0) * (rx + ry)));
  return s;
}

void set_params3d(pf_ctx* c, const pf_params* p) {
  pf::Implicit3DArgs& a = c->im;
  a.nx = (int)c->n[0];
  a.ny = (int)c->n[1];
  a.nz = (int)c->n[2];
  a.nf = c->nf;
  a.double_well = (c->model == PF_MODEL_AC);
  a.dw2 = (float)(2.0 * p->W);
  a.alpha = (float)p->fc_alpha;
  a.two_gamma = (float)(2.0 * p->fc_gamma);
  a.four_gamma = (float)(4.0 * p->fc_gamma);
  a.cb2g = (float)(p->fc_beta - 2.0 * p->fc_gamma);
  a.c3b6g = (float)(3.0 * p->fc_beta - 6.0 * p->fc_gamma);
  const double cell = c->h[0] * c->h[1] * c->h[2];
  for (int d = 0; d < 3; ++d) a.kg[d] = (float)(2.0 * p->kappa / (c->h[d] * c->h[d]));
  a.inv_dt = (float)(1.0 / p->dt);
  a.mob = (float)p->mobility;
  a.cell = (float)cell;
  a.unscaled = 0;
}

void destroy_graph(pf_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
  if (c->mob_graph) cudaGraphExecDestroy(c->mob_graph);
  c->mob_graph = nullptr;
}

// Captures the launches fn(stream) issues on the context's capture stream and
// instantiates them into *out.
template <class F>
pf_status capture_graph(pf_ctx* c, F&& fn, cudaGraphExec_t* out, const char* what) {
  if (!c->cap_stream) PF_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  PF_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  const cudaError_t le = fn(c->cap_stream);
  cudaGraph_t g = nullptr;
  const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
  if (le != cudaSuccess || ee != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, le != cudaSuccess ? le : ee, what);
  }
  const cudaError_t ie = cudaGraphInstantiate(out, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    *out = nullptr;
    return cuda_fail(c, ie, what);
  }
  return PF_OK;
}

// Executable graphs that live for one call (freed when their launches are done)
struct CallGraphs {
  cudaGraphExec_t g[3] = {nullptr, nullptr, nullptr};
  ~CallGraphs() {
    for (cudaGraphExec_t x : g)
      if (x) cudaGraphExecDestroy(x);
  }
};

cudaError_t launch_step(pf_ctx* c, const float* in, float* out, cudaStream_t s) {
  pf::Explicit2DArgs a = c->ex;
  a.in = in;
  a.out = out;
  a.pitch = pf::work_pitch((int)c->n[0]);
  return c->model == PF_MODEL_CH ? pf::launch_ch2d(a, s) : pf::launch_ac2d(a, s);
}

pf_status ensure_graph(pf_ctx* c) {
  if (c->graph) return PF_OK;
  if (!c->cap_stream) PF_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
  PF_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = cudaSuccess;
  for (int i = 0; i < kGraphSteps && le == cudaSuccess; ++i)
    le = (i % 2 == 0) ? launch_step(c, c->buf_a, c->buf_b, c->cap_stream)
                      : launch_step(c, c->buf_b, c->buf_a, c->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
  if (le != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return cuda_fail(c, le, "capture explicit steps");
  }
  if (ee != cudaSuccess) return cuda_fail(c, ee, "cudaStreamEndCapture");
  cudaError_t ie = cudaGraphInstantiate(&c->graph, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    c->graph = nullptr;
    return cuda_fail(c, ie, "cudaGraphInstantiate");
  }
  return PF_OK;
}

// ---- 2-D CH with a mobility field: plain-layout steps and the adjoint ------

int64_t nodes2d(const pf_ctx* c) { return c->n[0] * c->n[1]; }

// graph of kGraphSteps mobility-field steps buf_a -> buf_b -> ... -> buf_a
pf_status ensure_mob_graph(pf_ctx* c) {
  if (c->mob_graph && c->mob_graph_field == c->mob.mfield) return PF_OK;
  if (c->mob_graph) cudaGraphExecDestroy(c->mob_graph);
  c->mob_graph = nullptr;
  pf::ChMobArgs a = c->mob;
  const pf_status st = capture_graph(
      c,
      [&](cudaStream_t s) {
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < kGraphSteps && e == cudaSuccess; ++i) {
          a.d = (i % 2 == 0) ? c->buf_a : c->buf_b;
          e = pf::launch_ch_mob_step(a, (i % 2 == 0) ? c->buf_b : c->buf_a, s);
        }
        return e;
      },
      &c->mob_graph, "capture mobility-field steps");
  if (st == PF_OK) c->mob_graph_field = c->mob.mfield;
  return st;
}

// n steps from d_in into d_out (both plain planes) through the ping-pong
// planes; runs of kGraphSteps replay the mobility-field graph
pf_status mob_steps(pf_ctx* c, const float* d_in, float* d_out, int64_t n) {
  const int64_t N = nodes2d(c);
  if (n == 0) {
    if (d_out != d_in)
      PF_CUDA(cudaMemcpyAsync(d_out, d_in, sizeof(float) * N, cudaMemcpyDeviceToDevice, c->stream));
    return PF_OK;
  }
  const float* cur = d_in;
  if (n > kGraphSteps) {  // the last step still writes d_out directly
    pf_status st = ensure_mob_graph(c);
    if (st != PF_OK) return st;
    PF_CUDA(cudaMemcpyAsync(c->buf_a, d_in, sizeof(float) * N, cudaMemcpyDeviceToDevice,
                            c->stream));
    for (; n > kGraphSteps; n -= kGraphSteps) PF_CUDA(cudaGraphLaunch(c->mob_graph, c->stream));
    cur = c->buf_a;
  }
  pf::ChMobArgs a = c->mob;
  float* pp[2] = {c->buf_a, c->buf_b};
  int nxt = cur == c->buf_a ? 1 : 0;
  for (int64_t s = 0; s < n; ++s) {
    float* dst = (s == n - 1) ? d_out : pp[nxt];
    a.d = cur;
    PF_CUDA(pf::launch_ch_mob_step(a, dst, c->stream));
    cur = dst;
    nxt ^= 1;
  }
  return PF_OK;
}

pf_status step_explicit_mob(pf_ctx* c, float* state, int64_t n_steps) {
  const int64_t N = nodes2d(c);
  const float shift = (float)c->par.shift;
  float* cur = c->buf_a;
  float* oth = c->buf_b;
  PF_CUDA(pf::launch_add(state, cur, N, -shift, c->stream));
  int64_t left = n_steps;
  if (left >= kGraphSteps) {  // whole graphs leave the state in buf_a
    pf_status st = ensure_mob_graph(c);
    if (st != PF_OK) return st;
    for (; left >= kGraphSteps; left -= kGraphSteps) PF_CUDA(cudaGraphLaunch(c->mob_graph, c->stream));
  }
  pf::ChMobArgs a = c->mob;
  for (; left > 0; --left) {
    a.d = cur;
    PF_CUDA(pf::launch_ch_mob_step(a, oth, c->stream));
    std::swap(cur, oth);
  }
  PF_CUDA(pf::launch_add(cur, state, N, shift, c->stream));
  return PF_OK;
}

struct AdjLayout {
  size_t ck, seg, y0, y1, ones, ghi, glo, acc, small, total;
  int64_t nck;
};

AdjLayout adj_layout(const pf_ctx* c, int64_t n_steps, int ckpt) {
  AdjLayout L{};
  const size_t field = align_up(sizeof(float) * (size_t)nodes2d(c), 256);
  L.nck = (n_steps + ckpt - 1) / ckpt + 1;
  size_t off = 0;
  L.ck = off;
  off += field * L.nck;
  L.seg = off;
  off += field * ckpt;
  L.y0 = off;
  off += field;
  L.y1 = off;
  off += field;
  L.ones = off;
  off += field;
  L.ghi = off;  // running mobility gradient, a compensated FP32 pair per node
  off += field;
  L.glo = off;
  off += field;
  L.acc = off;
  off += align_up(sizeof(double) * 3 * pf::ch_mob_blocks((int)c->n[0], (int)c->n[1]), 256);
  L.small = off;
  off += align_up(sizeof(double) * 512, 256);
  L.total = off;
  return L;
}

// ---- batched ensembles of 2-D Allen-Cahn instances --------------------------

struct EnsLayout {
  std::vector<size_t> plane;  // offset of instance i's plane A (B follows)
  std::vector<size_t> plane_bytes;
  size_t args, tasks, offs, bar, total;
  int max_tasks;
};

int ens_tasks_for(int nx, int ny, int ty) {
  return ((nx + pf::kEnsOutCols - 1) / pf::kEnsOutCols) * ((ny + ty - 1) / ty);
}

EnsLayout ens_layout(const pf_ctx* c) {
  EnsLayout L;
  size_t off = 0;
  L.max_tasks = 0;
  for (int i = 0; i < c->ens_count; ++i) {
    const int nx = (int)c->ens_nx[i], ny = (int)c->ens_ny[i];
    const size_t b = align_up(sizeof(float) * (size_t)pf::work_pitch(nx) * pf::work_rows(ny), 256);
    L.plane.push_back(off);
    L.plane_bytes.push_back(b);
    off += 2 * b;
    L.max_tasks += ens_tasks_for(nx, ny, 6);
  }
  L.args = off;
  off += align_up(sizeof(pf::Explicit2DArgs) * c->ens_count, 256);
  L.tasks = off;
  off += align_up(sizeof(pf::EnsTask) * (size_t)L.max_tasks, 256);
  L.offs = off;
  off += align_up(sizeof(int64_t) * (c->ens_count + 1), 256);
  L.bar = off;
  off += 256;
  L.total = off;
  return L;
}

// Task list: every instance's (column strip, band) tasks, the tallest bands
// first so that the longest tasks start early (the order changes no result).
std::vector<pf::EnsTask> ens_build_tasks(const pf_ctx* c, const std::vector<int>& which) {
  std::vector<pf::EnsTask> t;
  for (int i : which) {
    const int nx = (int)c->ens_nx[i], ny = (int)c->ens_ny[i], ty = c->ens_ty[i];
    const int gx = (nx + pf::kEnsOutCols - 1) / pf::kEnsOutCols;
    for (int y0 = 0; y0 < ny; y0 += ty)
      for (int bx = 0; bx < gx; ++bx) t.push_back(pf::EnsTask{i, bx, y0, ty});
  }
  std::stable_sort(t.begin(), t.end(),
                   [](const pf::EnsTask& a, const pf::EnsTask& b) { return a.ty > b.ty; });
  return t;
}

pf_status ens_upload_tasks(pf_ctx* c, const std::vector<pf::EnsTask>& t) {
  c->ens_ntasks = (int)t.size();
  c->ens_host_tasks = t;
  PF_CUDA(cudaMemcpyAsync(c->ens_tasks, c->ens_host_tasks.data(), sizeof(pf::EnsTask) * t.size(),
                          cudaMemcpyHostToDevice, c->stream));
  PF_CUDA(cudaStreamSynchronize(c->stream));
  return PF_OK;
}

int ens_step_grid(int ntasks) {
  const int warps = pf::kEnsThreads / 32;
  return std::max(1, (ntasks + warps - 1) / warps);
}

// ---- 3-D: residual / JVP launches, explicit steps, Newton-GMRES -----------

pf_status check_ready(pf_ctx* c) {
  if (!c->ws) return fail(c, PF_ERR_STATE, "no workspace bound");
  if (!c->par_set) return fail(c, PF_ERR_STATE, "parameters not set");
  return PF_OK;
}

cudaError_t residual3d(pf_ctx* c, const float* U, const float* Un, float* out, int unscaled) {
  if (c->dim == 2) {
    pf::Implicit2DArgs a = c->im2;
    a.U = U;
    a.W = Un;
    a.out = out;
    a.unscaled = unscaled;
    return pf::launch_residual2d(a, c->stream);
  }
  pf::Implicit3DArgs a = c->im;
  a.U = U;
  a.W = Un;
  a.out = out;
  a.unscaled = unscaled;
  return pf::launch_residual3d(a, c->stream);
}

cudaError_t jvp3d(pf_ctx* c, const float* U, const float* v, float* out, int unscaled) {
  if (c->dim == 2) {
    pf::Implicit2DArgs a = c->im2;
    a.U = U;
    a.W = v;
    a.out = out;
    a.unscaled = unscaled;
    return pf::launch_jvp2d(a, c->stream);
  }
  pf::Implicit3DArgs a = c->im;
  a.U = U;
  a.W = v;
  a.out = out;
  a.unscaled = unscaled;
  return pf::launch_jvp3d(a, c->stream);
}

int64_t vec_len(const pf_ctx* c) { return nnodes(c) * imp_nf(c); }

// U <- U - dt G with G = L M^-1 r(U) (the residual with U^n = U)
pf_status step_explicit3d(pf_ctx* c, float* state, int64_t n_steps) {
  const int64_t n = vec_len(c);
  const float dt = (float)c->par.dt;
  for (int64_t s = 0; s < n_steps; ++s) {
    PF_CUDA(residual3d(c, state, state, c->g, 0));
    PF_CUDA(pf::launch_axpby(-dt, c->g, 1.0f, state, n, c->stream));
  }
  return PF_OK;
}

// ||M g||_2 in FP64 (weights = lumped mass), returned on the host
// The single-launch reductions need their block counter at 0: cleared once
// after every bind, then left at 0 by each reduction.
pf_status clear_count(pf_ctx* c) {
  if (!c->count_zeroed) {
    PF_CUDA(cudaMemsetAsync(c->count, 0, sizeof(unsigned), c->stream));
    c->count_zeroed = true;
  }
  return PF_OK;
}

pf_status mass_norm(pf_ctx* c, const float* g, double* out) {
  if (pf_status st = clear_count(c)) return st;
  PF_CUDA(pf::launch_mass_norm(g, (int)c->n[0], (int)c->n[1], (int)c->n[2], imp_nf(c),
                               c->h[0] * c->h[1] * c->h[2], c->partials, c->result, c->count,
                               c->stream));
  double h;
  PF_CUDA(cudaMemcpyAsync(&h, c->result, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PF_CUDA(cudaStreamSynchronize(c->stream));
  *out = std::sqrt(h);
  return PF_OK;
}

// Restarted GMRES(m) for (M^-1 J) x = -G at the linearisation point c->u, x in
// c->d (zero start), stopped at ||r|| <= max(rtol ||G||, atol).  Arnoldi with
// classical Gram-Schmidt applied twice (CGS2); inner products in FP64 on the
// device, Hessenberg and Givens rotations in FP64 on the host (Saad & Schultz
// 1986).
pf_status gmres3d(pf_ctx* c, int m, int maxit, double rtol, double atol, int* iters,
                  double* rel_out) {
  if (pf_status st = clear_count(c)) return st;
  const int64_t n = vec_len(c);
  const int64_t ldv = c->ldv;
  float* V = c->basis;
  double* dh1 = c->small;
  double* dh2 = c->small + pf::kMaxBasis;
  double* dnrm = c->small + 2 * pf::kMaxBasis;
  std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  double host[2 * pf::kMaxBasis + 1];
  PF_CUDA(cudaMemsetAsync(c->d, 0, sizeof(float) * n, c->stream));
  int total = 0;
  double beta0 = -1.0, rel = 1.0;
  for (;;) {
    // r = -G - J x  (x = 0 on the first cycle)
    if (total == 0) {
      PF_CUDA(pf::launch_axpby(-1.0f, c->g, 0.0f, V, n, c->stream));
    } else {
      PF_CUDA(jvp3d(c, c->u, c->d, V, 0));
      PF_CUDA(pf::launch_axpby(-1.0f, c->g, -1.0f, V, n, c->stream));
    }
    PF_CUDA(pf::launch_dots(V, ldv, 1, nullptr, n, c->partials, dnrm, c->count, c->stream));
    PF_CUDA(cudaMemcpyAsync(host, dnrm, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PF_CUDA(cudaStreamSynchronize(c->stream));
    const double beta = std::sqrt(host[0]);
    if (beta0 < 0) beta0 = beta;
    if (beta0 == 0.0) {
      rel = 0.0;
      break;
    }
    rel = beta / beta0;
    const double target = std::max(rtol * beta0, atol);
    if (beta <= target || total >= maxit) break;
    PF_CUDA(pf::launch_axpby((float)(1.0 / beta), V, 0.0f, V, n, c->stream));
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int k = 0;
    bool done = false;
    for (; k < m && total < maxit; ++k) {
      float* vk1 = V + (int64_t)(k + 1) * ldv;
      PF_CUDA(jvp3d(c, c->u, V + (int64_t)k * ldv, vk1, 0));
      PF_CUDA(pf::launch_dots(V, ldv, k + 1, vk1, n, c->partials, dh1, c->count, c->stream));
      PF_CUDA(pf::launch_update_dots(V, ldv, k + 1, dh1, vk1, n, c->partials, dh2, c->count,
                                       c->stream));
      PF_CUDA(pf::launch_update(V, ldv, k + 1, dh2, vk1, n, c->partials, dnrm, c->count, c->stream));
      PF_CUDA(cudaMemcpyAsync(host, c->small, sizeof(double) * (2 * pf::kMaxBasis + 1),
                              cudaMemcpyDeviceToHost, c->stream));
      PF_CUDA(cudaStreamSynchronize(c->stream));
      ++total;
      for (int j = 0; j <= k; ++j) H[(size_t)j * m + k] = host[j] + host[pf::kMaxBasis + j];
      const double hk1 = std::sqrt(std::max(host[2 * pf::kMaxBasis], 0.0));
      H[(size_t)(k + 1) * m + k] = hk1;
      if (hk1 > 0.0)
        PF_CUDA(pf::launch_axpby((float)(1.0 / hk1), vk1, 0.0f, vk1, n, c->stream));
      for (int j = 0; j < k; ++j) {
        const double t = cs[j] * H[(size_t)j * m + k] + sn[j] * H[(size_t)(j + 1) * m + k];
        H[(size_t)(j + 1) * m + k] = -sn[j] * H[(size_t)j * m + k] + cs[j] * H[(size_t)(j + 1) * m + k];
        H[(size_t)j * m + k] = t;
      }
      const double den = std::hypot(H[(size_t)k * m + k], hk1);
      cs[k] = den > 0 ? H[(size_t)k * m + k] / den : 1.0;
      sn[k] = den > 0 ? hk1 / den : 0.0;
      H[(size_t)k * m + k] = den;
      H[(size_t)(k + 1) * m + k] = 0.0;
      gv[k + 1] = -sn[k] * gv[k];
      gv[k] = cs[k] * gv[k];
      if (std::fabs(gv[k + 1]) <= target || hk1 == 0.0) {
        ++k;
        done = true;
        break;
      }
    }
    // y = H^-1 g (upper triangular), x += V y
    for (int i = k - 1; i >= 0; --i) {
      double s = gv[i];
      for (int j = i + 1; j < k; ++j) s -= H[(size_t)i * m + j] * y[j];
      y[i] = s / H[(size_t)i * m + i];
    }
    pf::LinComb lc{};
    for (int j = 0; j < k; ++j) lc.c[j] = (float)y[j];
    PF_CUDA(pf::launch_lincomb(V, ldv, k, lc, c->d, n, c->stream));
    if (done || total >= maxit) {
      rel = (k > 0) ? std::fabs(gv[k]) / beta0 : rel;
      break;
    }
  }
  *iters = total;
  *rel_out = rel;
  return PF_OK;
}

}  // namespace

extern "C" {

pf_status pf_create_mesh(pf_ctx** out, int dim, const int64_t nodes[3], const double h[3],
                         pf_model model, int n_fields, void* stream, size_t* workspace_bytes) {
  if (!out || !nodes || !h || !workspace_bytes) return PF_ERR_ARG;
  *out = nullptr;
  if (dim == 2) {  // explicit AC / CH, coupled AC-CH
    if (model == PF_MODEL_COUPLED) {
      if (n_fields != 2) return PF_ERR_ARG;
    } else {
      if (model != PF_MODEL_AC && model != PF_MODEL_CH) return PF_ERR_ARG;
      if (n_fields != 1) return PF_ERR_ARG;
    }
  } else if (dim == 3) {  // AC (double well, one field) or Fan-Chen (1..8 fields)
    if (model == PF_MODEL_AC) {
      if (n_fields != 1) return PF_ERR_ARG;
    } else if (model == PF_MODEL_FANCHEN) {
      if (n_fields < 1 || n_fields > 8) return PF_ERR_ARG;
    } else {
      return PF_ERR_ARG;
    }
  } else {
    return PF_ERR_ARG;
  }
  const int64_t minn = (model == PF_MODEL_CH || model == PF_MODEL_COUPLED) ? 3 : 2;
  int64_t total = 1;
  for (int k = 0; k < dim; ++k) {
    if (nodes[k] < minn || nodes[k] > (int64_t)1 << 20) return PF_ERR_ARG;
    if (!(h[k] > 0.0) || !isfinite(h[k])) return PF_ERR_ARG;
    total *= nodes[k];
    if (total > ((int64_t)1 << 31) - 1) return PF_ERR_ARG;
  }
  pf_ctx* c = new (std::nothrow) pf_ctx();
  if (!c) return PF_ERR_ARG;
  c->dim = dim;
  for (int k = 0; k < dim; ++k) {
    c->n[k] = nodes[k];
    c->h[k] = h[k];
  }
  c->model = model;
  c->nf = n_fields;
  c->stream = (cudaStream_t)stream;
  const Layout L = layout(c);
  c->ws_bytes = L.total;
  c->ws_explicit = L.explicit_total;
  *workspace_bytes = c->ws_bytes;
  *out = c;
  return PF_OK;
}

pf_status pf_explicit_workspace(const pf_ctx* c, size_t* bytes) {
  if (!c || !bytes) return PF_ERR_ARG;
  *bytes = c->ens_count > 0 ? c->ws_bytes : c->ws_explicit;
  return PF_OK;
}

pf_status pf_bind_workspace(pf_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c) return PF_ERR_ARG;
  if (!dev_ptr || (uintptr_t)dev_ptr % 256 != 0)
    return fail(c, PF_ERR_ARG, "workspace must be a non-null 256-byte aligned device pointer");
  const size_t need = c->ens_count > 0 ? c->ws_bytes : c->ws_explicit;
  if (bytes < need)
    return fail(c, PF_ERR_ARG, "workspace too small: %zu < %zu bytes", bytes, need);
  c->ws_bound = bytes;
  if (c->ens_count > 0) {
    const EnsLayout E = ens_layout(c);
    c->ws = (char*)dev_ptr;
    for (int i = 0; i < c->ens_count; ++i) {
      pf::Explicit2DArgs& x = c->ens_args[i];
      x.in = (float*)(c->ws + E.plane[i]);
      x.out = (float*)(c->ws + E.plane[i] + E.plane_bytes[i]);
    }
    c->ens_dargs = (pf::Explicit2DArgs*)(c->ws + E.args);
    c->ens_tasks = (pf::EnsTask*)(c->ws + E.tasks);
    c->ens_doff = (int64_t*)(c->ws + E.offs);
    c->ens_bar = (unsigned*)(c->ws + E.bar);
    destroy_graph(c);
    return PF_OK;
  }
  const Layout L = layout(c);
  c->ws = (char*)dev_ptr;
  c->partials = (double*)(c->ws + L.partials);
  c->result = (double*)(c->ws + L.result);
  c->count = (unsigned*)(c->ws + L.result + 128);
  c->count_zeroed = false;
  c->small = (double*)(c->ws + L.small);
  if (c->dim == 2) {
    c->buf_a = (float*)(c->ws + L.a);
    c->buf_b = (float*)(c->ws + L.b);
  }
  c->u = c->un = c->g = c->d = c->basis = nullptr;
  if (has_implicit(c)) {
    char* v = c->ws + L.vecs;
    if (bytes >= L.vecs + L.vec) c->g = (float*)v;
    if (implicit_bound(c)) {
      c->u = (float*)(v + L.vec);
      c->un = (float*)(v + 2 * L.vec);
      c->d = (float*)(v + 3 * L.vec);
      c->basis = (float*)(v + kVec3d * L.vec);
    }
    c->ldv = (int64_t)(L.vec / sizeof(float));
  }
  destroy_graph(c);
  return PF_OK;
}

// Coupled AC-CH (Eq. 7) with the Supp. 3 polynomials, coefficients of
// increasing powers: f_alpha(c), f_beta(c), h(eta).  The c polynomials are
// re-expanded about the shift s, in d = c - s, on the host in FP64.
void shift_poly(const double* a, int n, double s, double* out) {
  for (int k = 0; k < n; ++k) out[k] = 0.0;
  for (int j = 0; j < n; ++j) {  // a_j (s + d)^j = a_j sum_k C(j,k) s^(j-k) d^k
    double binom = 1.0;
    for (int k = 0; k <= j; ++k) {
      out[k] += a[j] * binom * std::pow(s, j - k);
      binom = binom * (j - k) / (k + 1);
    }
  }
}

void set_params_coupled(pf_ctx* c, const pf_params* p) {
  static const double fa[5] = {-1.6704, -4.776, 5.1622, -2.7375, 1.3687};
  static const double fb[3] = {-1.5924, -5.9746, 5.0};
  static const double h[6] = {0.0, 0.0, 0.0, 10.0, -15.0, 6.0};
  pf::Coupled2DArgs& a = c->cp;
  a.nx = (int)c->n[0];
  a.ny = (int)c->n[1];
  double sa[5], sb[3];
  shift_poly(fa, 5, p->shift, sa);
  shift_poly(fb, 3, p->shift, sb);
  for (int k = 0; k < 5; ++k) a.fa[k] = (float)sa[k];
  for (int k = 0; k < 4; ++k) a.dfa[k] = (float)((k + 1) * sa[k + 1]);
  for (int k = 0; k < 3; ++k) a.fb[k] = (float)sb[k];
  for (int k = 0; k < 2; ++k) a.dfb[k] = (float)((k + 1) * sb[k + 1]);
  for (int k = 0; k < 6; ++k) a.h[k] = (float)h[k];
  for (int k = 0; k < 5; ++k) a.dh[k] = (float)((k + 1) * h[k + 1]);
  const double hx = c->h[0], hy = c->h[1], m = hx * hy;
  a.k1 = stiffness2d(hx, hy, p->kappa / m);
  a.k2 = stiffness2d(hx, hy, -p->dt * p->mobility / m);
  a.neg_dt_meta = (float)(-p->dt * p->mobility2);
}

// The coupled step: working planes [c - shift; eta] without a frame in buf_a /
// buf_b (ping-pong), one fused launch per step.
pf_status step_coupled2d(pf_ctx* c, float* state, int64_t n_steps) {
  const int64_t N = nodes2d(c);
  const float shift = (float)c->par.shift;
  float* cur = c->buf_a;
  float* oth = c->buf_b;
  PF_CUDA(pf::launch_add(state, cur, N, -shift, c->stream));
  PF_CUDA(cudaMemcpyAsync(cur + N, state + N, sizeof(float) * N, cudaMemcpyDeviceToDevice,
                          c->stream));
  pf::Coupled2DArgs a = c->cp;
  for (int64_t s = 0; s < n_steps; ++s) {
    a.in = cur;
    a.out = oth;
    PF_CUDA(pf::launch_coupled2d(a, c->stream));
    std::swap(cur, oth);
  }
  PF_CUDA(pf::launch_add(cur, state, N, shift, c->stream));
  PF_CUDA(cudaMemcpyAsync(state + N, cur + N, sizeof(float) * N, cudaMemcpyDeviceToDevice,
                          c->stream));
  return PF_OK;
}

pf_status pf_set_form(pf_ctx* c, int form) {
  if (!c) return PF_ERR_ARG;
  if (form != PF_FORM_FUSED_GRAPH && form != PF_FORM_FUSED_STREAM && form != PF_FORM_TWO_PASS)
    return fail(c, PF_ERR_ARG, "unknown execution form %d", form);
  c->form = form;
  return PF_OK;
}

pf_status pf_set_params(pf_ctx* c, const pf_params* p) {
  if (!c) return PF_ERR_ARG;
  if (!p) return fail(c, PF_ERR_ARG, "params is NULL");
  if (!(p->dt > 0.0) || !(p->kappa >= 0.0) || !(p->mobility > 0.0) || !(p->W >= 0.0) ||
      !isfinite(p->dt) || !isfinite(p->kappa) || !isfinite(p->mobility) || !isfinite(p->W) ||
      !isfinite(p->shift))
    return fail(c, PF_ERR_ARG, "invalid parameters (need dt > 0, mobility > 0, kappa, W >= 0)");
  if (p->mobility_field && !(c->dim == 2 && c->model == PF_MODEL_CH))
    return fail(c, PF_ERR_ARG, "a per-node mobility field needs a 2-D Cahn-Hilliard mesh");
  if (c->model == PF_MODEL_COUPLED && (!(p->mobility2 > 0.0) || !isfinite(p->mobility2)))
    return fail(c, PF_ERR_ARG, "the coupled model needs mobility2 = M_eta > 0");
  c->par = *p;
  c->par_set = true;
  destroy_graph(c);
  if (c->dim == 3) {
    set_params3d(c, p);
    return PF_OK;
  }
  if (c->model == PF_MODEL_COUPLED) {
    set_params_coupled(c, p);
    return PF_OK;
  }
  if (c->model == PF_MODEL_AC || c->model == PF_MODEL_CH) {
    pf::Implicit2DArgs& b = c->im2;
    const double cell = c->h[0] * c->h[1];
    b.nx = (int)c->n[0];
    b.ny = (int)c->n[1];
    b.dw2 = (float)(2.0 * p->W);
    b.k = stiffness2d(c->h[0], c->h[1], p->kappa / cell);
    b.km = stiffness2d(c->h[0], c->h[1], p->mobility / cell);
    b.inv_dt = (float)(1.0 / p->dt);
    b.mob = (float)p->mobility;
    b.cell = (float)cell;
    b.unscaled = 0;
    b.ch = c->model == PF_MODEL_CH;
  }

  const double s = p->shift, W = p->W;
  // f'(s + d) = f'(s) + f''(s) d + f'''(s)/2 d^2 + f''''(s)/6 d^3 for f = W u^2 (1-u)^2
  double fp[4] = {W * (2 * s - 6 * s * s + 4 * s * s * s), W * (2 - 12 * s + 12 * s * s),
                  W * (-12 + 24 * s) / 2, 4 * W};
  const double hx = c->h[0], hy = c->h[1], m = hx * hy;
  pf::Explicit2DArgs& a = c->ex;
  a.nx = (int)c->n[0];
  a.ny = (int)c->n[1];
  if (c->model == PF_MODEL_AC) {
    const double f = -p->dt * p->mobility;
    a.p0 = (float)(f * fp[0] / 4);
    a.p1 = (float)(f * fp[1] / 4);
    a.p2 = (float)(f * fp[2] / 4);
    a.p3 = (float)(f * fp[3] / 4);
    a.k1 = stiffness2d(hx, hy, f * p->kappa / m);
    a.k2 = stiffness2d(hx, hy, 0.0);
  } else {
    a.p0 = (float)(fp[0] / 4);
    a.p1 = (float)(fp[1] / 4);
    a.p2 = (float)(fp[2] / 4);
    a.p3 = (float)(fp[3] / 4);
    a.k1 = stiffness2d(hx, hy, p->kappa / m);
    a.k2 = stiffness2d(hx, hy, -p->dt * p->mobility / m);
    pf::ChMobArgs& b = c->mob;
    b.nx = a.nx;
    b.ny = a.ny;
    b.mfield = p->mobility_field;
    b.p0 = (float)fp[0];
    b.p1 = (float)fp[1];
    b.p2 = (float)fp[2];
    b.p3 = (float)fp[3];
    // second derivative of f at s + d, expanded about s (exact quadratic in d)
    b.s0 = (float)(W * (2 - 12 * s + 12 * s * s));
    b.s1 = (float)(W * (-12 + 24 * s));
    b.s2 = (float)(12 * W);
    b.k = stiffness2d(hx, hy, 1.0 / m);
    b.kappa = (float)p->kappa;
    b.M = (float)p->mobility;
    b.W = (float)W;
    b.dt = (float)p->dt;
    b.ihx = (float)(1.0 / hx);
    b.ihy = (float)(1.0 / hy);
    b.cell = m;
  }
  pf::pack_explicit2d(a);
  destroy_graph(c);
  return PF_OK;
}

// The plain two-pass form: working planes without the ghost frame (buf_a,
// buf_b as nx x ny arrays), mu in the caller's state buffer meanwhile.
pf_status step_plain2d(pf_ctx* c, float* state, int64_t n_steps) {
  const int64_t N = nodes2d(c);
  const float shift = (float)c->par.shift;
  const bool ch = c->model == PF_MODEL_CH;
  float* cur = c->buf_a;
  float* oth = c->buf_b;
  PF_CUDA(pf::launch_add(state, cur, N, -shift, c->stream));
  for (int64_t s = 0; s < n_steps; ++s) {
    PF_CUDA(pf::launch_plain2d(ch, c->ex, cur, state, oth, c->stream));
    std::swap(cur, oth);
  }
  PF_CUDA(pf::launch_add(cur, state, N, shift, c->stream));
  return PF_OK;
}

pf_status pf_step_explicit(pf_ctx* c, float* state, int64_t n_steps) {
  if (!c) return PF_ERR_ARG;
  if (!c->ws) return fail(c, PF_ERR_STATE, "no workspace bound");
  if (!c->par_set) return fail(c, PF_ERR_STATE, "parameters not set");
  if (!state) return fail(c, PF_ERR_ARG, "state is NULL");
  if (n_steps < 0) return fail(c, PF_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return PF_OK;
  if (c->dim == 3) return step_explicit3d(c, state, n_steps);
  if (c->model == PF_MODEL_COUPLED) return step_coupled2d(c, state, n_steps);
  if (c->par.mobility_field) return step_explicit_mob(c, state, n_steps);
  if (c->form == PF_FORM_TWO_PASS) return step_plain2d(c, state, n_steps);
  const float shift = (float)c->par.shift;
  const int nx = (int)c->n[0], ny = (int)c->n[1];
  // working copies with the mirror frame: d = u - shift (both planes fully defined)
  PF_CUDA(pf::launch_to_work(state, c->buf_a, nx, ny, shift, c->stream));
  PF_CUDA(pf::launch_to_work(state, c->buf_b, nx, ny, shift, c->stream));
  int64_t left = n_steps;
  if (left >= kGraphSteps && c->form == PF_FORM_FUSED_GRAPH) {
    pf_status st = ensure_graph(c);
    if (st != PF_OK) return st;
    for (; left >= kGraphSteps; left -= kGraphSteps) PF_CUDA(cudaGraphLaunch(c->graph, c->stream));
  }
  float* cur = c->buf_a;
  float* oth = c->buf_b;
  for (; left > 0; --left) {
    PF_CUDA(launch_step(c, cur, oth, c->stream));
    float* t = cur;
    cur = oth;
    oth = t;
  }
  PF_CUDA(pf::launch_from_work(cur, state, nx, ny, shift, c->stream));
  return PF_OK;
}

pf_status pf_energy(pf_ctx* c, const float* state, double* energy, double* mass) {
  if (!c) return PF_ERR_ARG;
  if (!c->ws) return fail(c, PF_ERR_STATE, "no workspace bound");
  if (!c->par_set) return fail(c, PF_ERR_STATE, "parameters not set");
  if (!state) return fail(c, PF_ERR_ARG, "state is NULL");
  if (c->dim != 2) return fail(c, PF_ERR_ARG, "pf_energy supports 2-D meshes");
  if (c->model == PF_MODEL_COUPLED)
    return fail(c, PF_ERR_ARG, "pf_energy supports the AC and CH models");
  const double W = c->par.W;
  pf::Energy2DArgs a{};
  a.d = state;  // unshifted: f(u) = W (u^2 - 2 u^3 + u^4)
  a.nx = (int)c->n[0];
  a.ny = (int)c->n[1];
  a.hx = c->h[0];
  a.hy = c->h[1];
  a.shift = 0.0f;
  a.q0 = 0.0f;
  a.q1 = 0.0f;
  a.q2 = (float)W;
  a.q3 = (float)(-2 * W);
  a.q4 = (float)W;
  a.kappa = (float)c->par.kappa;
  PF_CUDA(pf::launch_energy2d(a, c->partials, c->result, c->stream));
  double host[2];
  PF_CUDA(cudaMemcpyAsync(host, c->result, sizeof(host), cudaMemcpyDeviceToHost, c->stream));
  PF_CUDA(cudaStreamSynchronize(c->stream));
  if (energy) *energy = host[0];
  if (mass) *mass = host[1];
  if (!isfinite(host[0]) || !isfinite(host[1]))
    return fail(c, PF_ERR_NONFINITE, "non-finite energy or mass (unstable time step?)");
  return PF_OK;
}

pf_status pf_step_implicit(pf_ctx* c, float* state, int64_t n_steps, const float* guess,
                           const pf_newton_opts* opts, pf_newton_stats* stats) {
  if (!c) return PF_ERR_ARG;
  pf_status st = check_ready(c);
  if (st != PF_OK) return st;
  if (!has_implicit(c))
    return fail(c, PF_ERR_ARG, "pf_step_implicit supports 3-D meshes and 2-D AC / CH");
  if ((st = need_implicit_ws(c)) != PF_OK) return st;
  if (!state) return fail(c, PF_ERR_ARG, "state is NULL");
  if (c->par.mobility_field)
    return fail(c, PF_ERR_ARG, "pf_step_implicit has no per-node mobility field");
  if (n_steps < 0) return fail(c, PF_ERR_ARG, "n_steps < 0");
  pf_newton_opts o{20, 30, 300, 1e-5, 1e-3};
  if (opts) o = *opts;
  if (o.gmres_restart < 1 || o.gmres_restart > pf::kMaxBasis - 1 || o.max_newton < 0 ||
      o.gmres_max_iters < 1 || !(o.newton_rtol > 0) || !(o.gmres_rtol > 0))
    return fail(c, PF_ERR_ARG, "invalid Newton/GMRES options (restart must be 1..%d)",
                pf::kMaxBasis - 1);
  pf_newton_stats s{0, 0, 1, 0.0, 0.0};
  const int64_t n = vec_len(c);
  const double inv_dt = 1.0 / c->par.dt;
  const int64_t n_state = split_ch(c) ? nnodes(c) : n;  // CH: the state is c alone
  for (int64_t step = 0; step < n_steps; ++step) {
    PF_CUDA(cudaMemcpyAsync(c->un, state, sizeof(float) * n_state, cudaMemcpyDeviceToDevice,
                            c->stream));
    const float* start = (step == 0 && guess) ? guess : state;
    PF_CUDA(cudaMemcpyAsync(c->u, start, sizeof(float) * n_state, cudaMemcpyDeviceToDevice,
                            c->stream));
    if (split_ch(c)) {
      // mu of the starting c: with mu = 0 the mu row of M^-1 R is -M^-1 r(c)
      const int64_t N = nnodes(c);
      PF_CUDA(cudaMemsetAsync(c->un + N, 0, sizeof(float) * N, c->stream));
      PF_CUDA(cudaMemsetAsync(c->u + N, 0, sizeof(float) * N, c->stream));
      PF_CUDA(residual3d(c, c->u, c->un, c->g, 0));
      PF_CUDA(pf::launch_axpby(-1.0f, c->g + N, 0.0f, c->u + N, N, c->stream));
    }
    double ref;
    st = mass_norm(c, c->un, &ref);  // ||M U^n||; the target is rtol ||M U^n / dt||
    if (st != PF_OK) return st;
    const double tol = o.newton_rtol * ref * inv_dt;
    // No oversolving: a linear residual below a tenth of Newton's target (in
    // the M-norm; GMRES measures the Euclidean norm of M^-1 R, and
    // ||v||_M <= sqrt(h^3) ||v||_2 for the lumped mass) is as good as exact.
    const double atol = kNoOversolve * tol / std::sqrt(c->h[0] * c->h[1] * c->h[2]);
    bool ok = false;
    double rn = 0.0;
    for (int it = 0;; ++it) {
      PF_CUDA(residual3d(c, c->u, c->un, c->g, 0));
      st = mass_norm(c, c->g, &rn);
      if (st != PF_OK) return st;
      if (!std::isfinite(rn)) return fail(c, PF_ERR_NONFINITE, "non-finite Newton residual");
      if (step == 0 && it == 0) s.initial_residual = rn;
      if (rn <= tol) {
        ok = true;
        break;
      }
      if (it >= o.max_newton) break;
      int gi = 0;
      double rel = 0.0;
      st = gmres3d(c, o.gmres_restart, o.gmres_max_iters, o.gmres_rtol, atol, &gi, &rel);
      if (st != PF_OK) return st;
      s.gmres_iters += gi;
      s.newton_iters += 1;
      PF_CUDA(pf::launch_axpby(1.0f, c->d, 1.0f, c->u, n, c->stream));
    }
    s.final_residual = rn;
    if (!ok) s.converged = 0;
    PF_CUDA(cudaMemcpyAsync(state, c->u, sizeof(float) * n_state, cudaMemcpyDeviceToDevice,
                            c->stream));
    if (!ok) {
      PF_CUDA(cudaStreamSynchronize(c->stream));
      if (stats) *stats = s;
      return fail(c, PF_ERR_NOT_CONVERGED, "Newton did not reach ||R|| <= %g (got %g) in step %lld",
                  tol, rn, (long long)step);
    }
  }
  PF_CUDA(cudaStreamSynchronize(c->stream));
  if (stats) *stats = s;
  return PF_OK;
}

pf_status pf_create_ensemble(pf_ctx** out, int count, const int64_t* nx, const int64_t* ny,
                             const double* h, void* stream, size_t* workspace_bytes,
                             int64_t* offsets) {
  if (!out || !nx || !ny || !workspace_bytes || count < 1 || count > (1 << 20)) return PF_ERR_ARG;
  *out = nullptr;
  int64_t total = 0;
  for (int i = 0; i < count; ++i) {
    if (nx[i] < 4 || ny[i] < 4 || nx[i] > (1 << 20) || ny[i] > (1 << 20)) return PF_ERR_ARG;
    if (h && (!(h[2 * i] > 0) || !(h[2 * i + 1] > 0))) return PF_ERR_ARG;
    total += nx[i] * ny[i];
    if (total > ((int64_t)1 << 33)) return PF_ERR_ARG;
  }
  pf_ctx* c = new (std::nothrow) pf_ctx();
  if (!c) return PF_ERR_ARG;
  c->dim = 2;
  c->model = PF_MODEL_AC;
  c->nf = 1;
  c->stream = (cudaStream_t)stream;
  c->ens_count = count;
  c->ens_off.push_back(0);
  for (int i = 0; i < count; ++i) {
    c->ens_nx.push_back(nx[i]);
    c->ens_ny.push_back(ny[i]);
    c->ens_hx.push_back(h ? h[2 * i] : 1.0);
    c->ens_hy.push_back(h ? h[2 * i + 1] : 1.0);
    c->ens_ty.push_back(12);
    c->ens_off.push_back(c->ens_off.back() + nx[i] * ny[i]);
    pf::Explicit2DArgs x{};
    x.nx = (int)nx[i];
    x.ny = (int)ny[i];
    x.pitch = pf::work_pitch(x.nx);
    x.rows = pf::work_rows(x.ny);
    c->ens_args.push_back(x);
  }
  c->n[0] = nx[0];
  c->n[1] = ny[0];
  c->ws_bytes = ens_layout(c).total;
  *workspace_bytes = c->ws_bytes;
  if (offsets)
    for (int i = 0; i <= count; ++i) offsets[i] = c->ens_off[i];
  *out = c;
  return PF_OK;
}

pf_status pf_set_ensemble_params(pf_ctx* c, const pf_params* p) {
  if (!c) return PF_ERR_ARG;
  if (c->ens_count < 1) return fail(c, PF_ERR_ARG, "not an ensemble context");
  if (!c->ws) return fail(c, PF_ERR_STATE, "no workspace bound");
  if (!p) return fail(c, PF_ERR_ARG, "params is NULL");
  c->ens_iso = true;
  for (int i = 0; i < c->ens_count; ++i) {
    const pf_params& q = p[i];
    if (!(q.dt > 0.0) || !(q.kappa >= 0.0) || !(q.mobility > 0.0) || !(q.W >= 0.0) ||
        !std::isfinite(q.dt) || !std::isfinite(q.kappa) || !std::isfinite(q.mobility) ||
        !std::isfinite(q.W) || !std::isfinite(q.shift) || q.mobility_field)
      return fail(c, PF_ERR_ARG, "invalid parameters for instance %d", i);
    if (q.shift != p[0].shift) return fail(c, PF_ERR_ARG, "all instances must share one shift");
    pf::Explicit2DArgs& a = c->ens_args[i];
    const double s = q.shift, W = q.W, hx = c->ens_hx[i], hy = c->ens_hy[i], m = hx * hy;
    const double fp[4] = {W * (2 * s - 6 * s * s + 4 * s * s * s), W * (2 - 12 * s + 12 * s * s),
                          W * (-12 + 24 * s) / 2, 4 * W};
    const double f = -q.dt * q.mobility;
    a.p0 = (float)(f * fp[0] / 4);
    a.p1 = (float)(f * fp[1] / 4);
    a.p2 = (float)(f * fp[2] / 4);
    a.p3 = (float)(f * fp[3] / 4);
    a.k1 = stiffness2d(hx, hy, f * q.kappa / m);
    a.k2 = stiffness2d(hx, hy, 0.0);
    pf::pack_explicit2d(a);
    if (!(a.k1.cx == a.k1.cd && a.k1.cy == a.k1.cd)) c->ens_iso = false;
  }
  c->par = p[0];
  c->par_set = true;
  PF_CUDA(cudaMemcpyAsync(c->ens_dargs, c->ens_args.data(),
                          sizeof(pf::Explicit2DArgs) * c->ens_count, cudaMemcpyHostToDevice,
                          c->stream));
  PF_CUDA(cudaMemcpyAsync(c->ens_doff, c->ens_off.data(), sizeof(int64_t) * (c->ens_count + 1),
                          cudaMemcpyHostToDevice, c->stream));
  std::vector<int> all(c->ens_count);
  for (int i = 0; i < c->ens_count; ++i) all[i] = i;
  return ens_upload_tasks(c, ens_build_tasks(c, all));
}

// Schedule candidates of an instance: band height kEnsTy[j % 3] and L2
// policy j / 3 (pf::kL2Normal, kL2Stream, kL2StreamHalf).
constexpr int kEnsTy[3] = {6, 12, 24};
constexpr int kEnsCands = 9;

// Upload the per-instance arguments and the task list for the current
// schedule (synchronises the stream).
pf_status ens_upload_schedule(pf_ctx* c) {
  PF_CUDA(cudaMemcpyAsync(c->ens_dargs, c->ens_args.data(),
                          sizeof(pf::Explicit2DArgs) * c->ens_count, cudaMemcpyHostToDevice,
                          c->stream));
  std::vector<int> all(c->ens_count);
  for (int i = 0; i < c->ens_count; ++i) all[i] = i;
  return ens_upload_tasks(c, ens_build_tasks(c, all));
}

pf_status pf_set_ensemble_schedule(pf_ctx* c, const int* ty, const int* l2) {
  if (!c) return PF_ERR_ARG;
  if (c->ens_count < 1) return fail(c, PF_ERR_ARG, "not an ensemble context");
  if (!c->ws || !c->par_set) return fail(c, PF_ERR_STATE, "workspace or parameters missing");
  for (int i = 0; i < c->ens_count; ++i) {
    if (ty && ty[i] != 6 && ty[i] != 12 && ty[i] != 24)
      return fail(c, PF_ERR_ARG, "band height of instance %d is not 6, 12 or 24", i);
    if (l2 && (l2[i] < pf::kL2Normal || l2[i] > pf::kL2StreamHalf))
      return fail(c, PF_ERR_ARG, "L2 policy of instance %d is not 0, 1 or 2", i);
  }
  for (int i = 0; i < c->ens_count; ++i) {
    if (ty) c->ens_ty[i] = ty[i];
    if (l2) c->ens_args[i].l2 = l2[i];
  }
  destroy_graph(c);
  return ens_upload_schedule(c);
}

pf_status pf_tune_ensemble(pf_ctx* c, int reps, int* ty_out, int* l2_out, double* us_out) {
  if (!c) return PF_ERR_ARG;
  if (c->ens_count < 1) return fail(c, PF_ERR_ARG, "not an ensemble context");
  if (!c->ws || !c->par_set) return fail(c, PF_ERR_STATE, "workspace or parameters missing");
  if (reps < 1) return fail(c, PF_ERR_ARG, "reps must be >= 1");
  // planes hold defined values while timing (the step is data-independent in cost)
  for (int i = 0; i < c->ens_count; ++i) {
    const pf::Explicit2DArgs& x = c->ens_args[i];
    PF_CUDA(cudaMemsetAsync(const_cast<float*>(x.in), 0, sizeof(float) * x.pitch * x.rows, c->stream));
    PF_CUDA(cudaMemsetAsync(x.out, 0, sizeof(float) * x.pitch * x.rows, c->stream));
  }
  std::vector<std::pair<int64_t, int64_t>> classes;
  std::vector<int> cls(c->ens_count);
  for (int i = 0; i < c->ens_count; ++i) {
    auto k = std::make_pair(c->ens_nx[i], c->ens_ny[i]);
    auto it = std::find(classes.begin(), classes.end(), k);
    cls[i] = (int)(it - classes.begin());
    if (it == classes.end()) classes.push_back(k);
  }
  const int nc = (int)classes.size();
  cudaEvent_t e0, e1;
  PF_CUDA(cudaEventCreate(&e0));
  PF_CUDA(cudaEventCreate(&e1));
  // whole-ensemble step time (us, best of three rounds of `reps` per-step
  // launches) with candidate assign[class] for every instance of a class; the
  // rounds run back to back, so the later ones see the L2 contents the
  // schedule leaves from step to step
  auto time_all = [&](const std::vector<int>& assign, double* us) -> pf_status {
    for (int i = 0; i < c->ens_count; ++i) {
      c->ens_ty[i] = kEnsTy[assign[cls[i]] % 3];
      c->ens_args[i].l2 = assign[cls[i]] / 3;
    }
    pf_status s = ens_upload_schedule(c);
    if (s != PF_OK) return s;
    const int grid = ens_step_grid(c->ens_ntasks);
    double best = 1e30;
    for (int round = 0; round < 3; ++round) {
      cudaError_t e = pf::launch_ensemble_step(c->ens_tasks, c->ens_ntasks, c->ens_dargs, 0,
                                               c->ens_iso, grid, c->stream);  // warm-up
      if (e == cudaSuccess) e = cudaEventRecord(e0, c->stream);
      for (int r = 0; r < reps && e == cudaSuccess; ++r)
        e = pf::launch_ensemble_step(c->ens_tasks, c->ens_ntasks, c->ens_dargs, (r + 1) & 1,
                                     c->ens_iso, grid, c->stream);
      if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) return cuda_fail(c, e, "ensemble tuning");
      best = std::min(best, 1e3 * ms / reps);
    }
    *us = best;
    return PF_OK;
  };
  pf_status st = PF_OK;
  // 1. every class on the same candidate
  double uni[kEnsCands];
  int bj = 0;
  for (int j = 0; j < kEnsCands && st == PF_OK; ++j) {
    st = time_all(std::vector<int>(nc, j), &uni[j]);
    if (st == PF_OK && uni[j] < uni[bj]) bj = j;
  }
  std::vector<int> assign(nc, bj);
  double best = st == PF_OK ? uni[bj] : 0.0;
  if (us_out)
    for (int ci = 0; ci < nc; ++ci)
      for (int j = 0; j < kEnsCands; ++j) us_out[kEnsCands * ci + j] = j == bj ? best : -1.0;
  // 2. coordinate descent over the classes, most nodes first (the classes
  // that fill L2 the most are the first to try streaming): a class keeps
  // another candidate only if the whole step gets at least 1 % faster
  std::vector<int> order(nc);
  for (int ci = 0; ci < nc; ++ci) order[ci] = ci;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return classes[x].first * classes[x].second > classes[y].first * classes[y].second;
  });
  for (int pass = 0; pass < 3 && st == PF_OK; ++pass) {
    bool changed = false;
    for (int ci : order) {
      for (int j = 0; j < kEnsCands && st == PF_OK; ++j) {
        if (j == assign[ci]) continue;
        std::vector<int> trial = assign;
        trial[ci] = j;
        double t = 0.0;
        st = time_all(trial, &t);
        if (st != PF_OK) break;
        if (us_out) us_out[kEnsCands * ci + j] = t;
        if (t < 0.99 * best) {
          best = t;
          assign = trial;
          changed = true;
        }
      }
      if (st != PF_OK) break;
    }
    if (!changed) break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != PF_OK) return st;
  if (us_out) {
    for (int j = 0; j < kEnsCands; ++j) us_out[kEnsCands * nc + j] = uni[j];
    us_out[kEnsCands * nc + kEnsCands] = best;
  }
  for (int i = 0; i < c->ens_count; ++i) {
    c->ens_ty[i] = kEnsTy[assign[cls[i]] % 3];
    c->ens_args[i].l2 = assign[cls[i]] / 3;
    if (ty_out) ty_out[i] = c->ens_ty[i];
    if (l2_out) l2_out[i] = c->ens_args[i].l2;
  }
  destroy_graph(c);
  return ens_upload_schedule(c);
}

pf_status pf_step_ensemble(pf_ctx* c, float* packed, int64_t n_steps, int mode) {
  if (!c) return PF_ERR_ARG;
  if (c->ens_count < 1) return fail(c, PF_ERR_ARG, "not an ensemble context");
  if (!c->ws || !c->par_set) return fail(c, PF_ERR_STATE, "workspace or parameters missing");
  if (!packed) return fail(c, PF_ERR_ARG, "state is NULL");
  if (n_steps < 0 || n_steps > INT32_MAX) return fail(c, PF_ERR_ARG, "bad n_steps");
  if (mode < PF_ENS_PERSISTENT || mode > PF_ENS_PLAIN) return fail(c, PF_ERR_ARG, "bad mode");
  if (n_steps == 0) return PF_OK;
  const float shift = (float)c->par.shift;
  PF_CUDA(pf::launch_ens_to_work(packed, c->ens_doff, c->ens_dargs, c->ens_count, shift, c->stream));
  if (mode == PF_ENS_PERSISTENT) {
    const int grid = pf::ensemble_persistent_grid(c->ens_iso);
    if (grid < 1) return fail(c, PF_ERR_CUDA, "cannot size the persistent grid");
    PF_CUDA(cudaMemsetAsync(c->ens_bar, 0, 3 * sizeof(unsigned), c->stream));
    // one persistent launch for all steps, recorded as a one-node CUDA graph
    if (!c->cap_stream) PF_CUDA(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    PF_CUDA(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    cudaError_t le = pf::launch_ensemble_persistent(c->ens_tasks, c->ens_ntasks, c->ens_dargs,
                                                    (int)n_steps, c->ens_bar, 2000000000LL,
                                                    c->ens_iso, grid, c->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &g);
    if (le != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      return cuda_fail(c, le != cudaSuccess ? le : ee, "capture persistent ensemble launch");
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return cuda_fail(c, ie, "instantiate persistent ensemble graph");
    cudaError_t re = cudaGraphLaunch(ex, c->stream);
    cudaGraphExecDestroy(ex);
    if (re != cudaSuccess) return cuda_fail(c, re, "launch persistent ensemble graph");
  } else if (mode == PF_ENS_PER_STEP) {
    const int grid = ens_step_grid(c->ens_ntasks);
    for (int64_t s = 0; s < n_steps; ++s)
      PF_CUDA(pf::launch_ensemble_step(c->ens_tasks, c->ens_ntasks, c->ens_dargs, (int)(s & 1),
                                       c->ens_iso, grid, c->stream));
  } else {  // plain: the single-instance fused step, one launch per instance and step
    for (int64_t s = 0; s < n_steps; ++s)
      for (int i = 0; i < c->ens_count; ++i) {
        pf::Explicit2DArgs a = c->ens_args[i];
        if (s & 1) {
          a.in = a.out;
          a.out = const_cast<float*>(c->ens_args[i].in);
        }
        PF_CUDA(pf::launch_ac2d(a, c->stream));
      }
  }
  PF_CUDA(pf::launch_ens_from_work(packed, c->ens_doff, c->ens_dargs, c->ens_count,
                                   (int)(n_steps & 1), shift, c->stream));
  if (mode == PF_ENS_PERSISTENT) {
    unsigned flag = 0;
    PF_CUDA(cudaMemcpyAsync(&flag, c->ens_bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost,
                            c->stream));
    PF_CUDA(cudaStreamSynchronize(c->stream));
    if (flag) return fail(c, PF_ERR_TIMEOUT, "grid barrier wait expired in the persistent ensemble");
  }
  return PF_OK;
}

pf_status pf_barrier_selftest(unsigned* dev_scratch, long long limit_cycles, int phantom,
                              void* stream) {
  if (!dev_scratch || limit_cycles < 1 || phantom < 0 || phantom > 1) return PF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  if (cudaMemsetAsync(dev_scratch, 0, 3 * sizeof(unsigned), s) != cudaSuccess) return PF_ERR_CUDA;
  if (pf::launch_barrier_selftest(dev_scratch, limit_cycles, phantom, s) != cudaSuccess)
    return PF_ERR_CUDA;
  unsigned flag = 0;
  if (cudaMemcpyAsync(&flag, dev_scratch + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, s) !=
          cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return PF_ERR_CUDA;
  return flag ? PF_ERR_TIMEOUT : PF_OK;
}

// ---- adjoint of an implicit trajectory (Supp. 2, Eq. II.1-II.6) ----------

size_t iadj_vec(const pf_ctx* c) { return align_up(sizeof(float) * (size_t)vec_len(c), 256); }

bool iadj_ok(const pf_ctx* c) { return has_implicit(c) && !split_ch(c); }

// out = L K U (unscaled): the residual with no local energy and kappa = 1 at U^n = U
cudaError_t stiff_only(pf_ctx* c, const float* U, float* out) {
  if (c->dim == 2) {
    pf::Implicit2DArgs a = c->im2;
    a.dw2 = 0.0f;
    a.k = stiffness2d(c->h[0], c->h[1], 1.0 / (c->h[0] * c->h[1]));
    a.U = U;
    a.W = U;
    a.out = out;
    a.unscaled = 1;
    return pf::launch_residual2d(a, c->stream);
  }
  pf::Implicit3DArgs a = c->im;
  a.dw2 = 0.0f;
  a.alpha = a.two_gamma = a.four_gamma = a.cb2g = a.c3b6g = 0.0f;
  for (int d = 0; d < 3; ++d) a.kg[d] = (float)(2.0 / (c->h[d] * c->h[d]));  // kappa = 1
  a.U = U;
  a.W = U;
  a.out = out;
  a.unscaled = 1;
  return pf::launch_residual3d(a, c->stream);
}

// FP64 dot product of two device vectors of the context's length, on the host
pf_status dot_host(pf_ctx* c, const float* a, const float* b, double* scratch, double* out) {
  if (pf_status st = clear_count(c)) return st;
  PF_CUDA(pf::launch_dots(a, 0, 1, b, vec_len(c), c->partials, scratch, c->count, c->stream));
  PF_CUDA(cudaMemcpyAsync(out, scratch, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PF_CUDA(cudaStreamSynchronize(c->stream));
  return PF_OK;
}

pf_status pf_adjoint_workspace(pf_ctx* c, int64_t n_steps, int ckpt_every, size_t* bytes) {
  if (!c || !bytes) return PF_ERR_ARG;
  if (c->dim != 2 || c->model != PF_MODEL_CH)
    return fail(c, PF_ERR_ARG, "the adjoint needs a 2-D Cahn-Hilliard mesh");
  if (n_steps < 1 || ckpt_every < 1) return fail(c, PF_ERR_ARG, "n_steps and ckpt_every must be >= 1");
  *bytes = adj_layout(c, n_steps, ckpt_every).total;
  return PF_OK;
}

pf_status pf_adjoint(pf_ctx* c, const float* state0, const float* target, int64_t n_steps,
                     int ckpt_every, int nodal_loss, void* adj_ws, size_t adj_bytes, double* loss,
                     double* grad_scalars, double* grad_mobility, float* grad_state0) {
  if (!c) return PF_ERR_ARG;
  pf_status st = check_ready(c);
  if (st != PF_OK) return st;
  if (c->dim != 2 || c->model != PF_MODEL_CH)
    return fail(c, PF_ERR_ARG, "the adjoint needs a 2-D Cahn-Hilliard mesh");
  if (!state0 || !target || !adj_ws) return fail(c, PF_ERR_ARG, "null array");
  if (n_steps < 1 || ckpt_every < 1) return fail(c, PF_ERR_ARG, "n_steps and ckpt_every must be >= 1");
  const AdjLayout L = adj_layout(c, n_steps, ckpt_every);
  if (adj_bytes < L.total || (uintptr_t)adj_ws % 256)
    return fail(c, PF_ERR_ARG, "adjoint workspace too small or misaligned (%zu < %zu)", adj_bytes,
                L.total);
  const int nx = (int)c->n[0], ny = (int)c->n[1];
  const int64_t N = nodes2d(c);
  const size_t field = align_up(sizeof(float) * (size_t)N, 256);
  char* ws = (char*)adj_ws;
  auto ck = [&](int64_t i) { return (float*)(ws + L.ck + field * i); };
  auto seg = [&](int64_t i) { return (float*)(ws + L.seg + field * i); };
  float* y0 = (float*)(ws + L.y0);
  float* y1 = (float*)(ws + L.y1);
  float* ones = (float*)(ws + L.ones);
  double* acc = (double*)(ws + L.acc);
  double* small = (double*)(ws + L.small);
  float* ghi = grad_mobility ? (float*)(ws + L.ghi) : nullptr;
  float* glo = grad_mobility ? (float*)(ws + L.glo) : nullptr;
  const int nb = pf::ch_mob_blocks(nx, ny);
  const float shift = (float)c->par.shift;
  const double cell = c->h[0] * c->h[1];
  const float* saved_field = c->mob.mfield;
  if (!c->mob.mfield) {  // uniform mobility: a field of ones
    PF_CUDA(cudaMemsetAsync(ones, 0, sizeof(float) * N, c->stream));
    PF_CUDA(pf::launch_add(ones, ones, N, 1.0f, c->stream));
    c->mob.mfield = ones;
  }
  pf::ChMobArgs a = c->mob;
  a.ngm = (float)(-(double)a.dt * a.M * a.cell);
  // forward with checkpoints: ck(j) = d^{j * ckpt_every}, ck(last) = d^N
  const int64_t last = (n_steps + ckpt_every - 1) / ckpt_every;
  PF_CUDA(pf::launch_add(state0, ck(0), N, -shift, c->stream));
  for (int64_t j = 0; j < last && st == PF_OK; ++j) {
    const int64_t len = std::min<int64_t>(ckpt_every, n_steps - j * ckpt_every);
    st = mob_steps(c, ck(j), ck(j + 1), len);
  }
  if (st == PF_OK) {
    PF_CUDA(pf::launch_loss(ck(last), shift, target, nx, ny, cell, nodal_loss, y0, small + 8,
                            small, c->stream));
    PF_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 3 * nb, c->stream));
    if (grad_mobility) {
      PF_CUDA(cudaMemsetAsync(ghi, 0, sizeof(float) * N, c->stream));
      PF_CUDA(cudaMemsetAsync(glo, 0, sizeof(float) * N, c->stream));
    }
    float* yin = y0;
    float* yout = y1;
    // whole segments replay graphs captured here (while the forward pass runs):
    // g[0] recomputes seg(1 .. ckpt-1) from seg(0), g[1 + p] reverses a segment
    // starting from y0 (p = 0) or y1 (p = 1); a shorter last segment launches
    // its steps one by one
    CallGraphs cg;
    const bool graphs = ckpt_every >= 8;
    auto recompute = [&](cudaStream_t s, int64_t len) {
      pf::ChMobArgs r = a;
      cudaError_t e = cudaSuccess;
      for (int64_t t = 1; t < len && e == cudaSuccess; ++t) {
        r.d = seg(t - 1);
        e = pf::launch_ch_mob_step(r, seg(t), s);
      }
      return e;
    };
    auto reverse = [&](cudaStream_t s, int64_t len, float* yi, float* yo) {
      pf::ChMobArgs r = a;
      cudaError_t e = cudaSuccess;
      for (int64_t t = len - 1; t >= 0 && e == cudaSuccess; --t) {
        r.d = seg(t);
        e = pf::launch_ch_adj_step(r, yi, yo, ghi, glo, acc, s);
        std::swap(yi, yo);
      }
      return e;
    };
    for (int64_t j = last - 1; j >= 0 && st == PF_OK; --j) {
      const int64_t start = j * ckpt_every;
      const int64_t len = std::min<int64_t>(ckpt_every, n_steps - start);
      const bool whole = graphs && len == ckpt_every;
      // recompute d^{start} .. d^{start+len-1} into the segment buffer
      PF_CUDA(cudaMemcpyAsync(seg(0), ck(j), sizeof(float) * N, cudaMemcpyDeviceToDevice,
                              c->stream));
      cudaError_t e = cudaSuccess;
      if (whole) {
        if (!cg.g[0])
          st = capture_graph(c, [&](cudaStream_t s) { return recompute(s, ckpt_every); }, &cg.g[0],
                             "capture the recompute");
        if (st == PF_OK) e = cudaGraphLaunch(cg.g[0], c->stream);
        const int p = yin == y0 ? 0 : 1;
        if (st == PF_OK && e == cudaSuccess && !cg.g[1 + p])
          st = capture_graph(c, [&](cudaStream_t s) { return reverse(s, ckpt_every, yin, yout); },
                             &cg.g[1 + p], "capture the reverse sweep");
        if (st == PF_OK && e == cudaSuccess) e = cudaGraphLaunch(cg.g[1 + p], c->stream);
        if (ckpt_every % 2) std::swap(yin, yout);
      } else {
        e = recompute(c->stream, len);
        if (e == cudaSuccess) e = reverse(c->stream, len, yin, yout);
        if (len % 2) std::swap(yin, yout);
      }
      if (st == PF_OK && e != cudaSuccess) {
        c->mob.mfield = saved_field;
        return cuda_fail(c, e, "adjoint step");
      }
    }
    if (st == PF_OK) {
      cudaError_t e = pf::launch_colsum(acc, nb, 3, 3, small + 1, c->stream);
      if (e == cudaSuccess && grad_mobility)
        e = pf::launch_grad_to_double(ghi, glo, grad_mobility, N, c->stream);
      if (e == cudaSuccess && grad_state0)
        e = pf::launch_mass_scale(yin, nx, ny, cell, grad_state0, c->stream);
      double host[4] = {0, 0, 0, 0};
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(host, small, sizeof(host), cudaMemcpyDeviceToHost, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) {
        c->mob.mfield = saved_field;
        return cuda_fail(c, e, "adjoint reductions");
      }
      if (loss) *loss = host[0];
      if (grad_scalars) {
        grad_scalars[0] = host[1];
        grad_scalars[1] = host[2];
        grad_scalars[2] = host[3];
      }
      if (!std::isfinite(host[0])) st = fail(c, PF_ERR_NONFINITE, "non-finite loss");
    }
  }
  c->mob.mfield = saved_field;
  return st;
}

pf_status pf_jvp(pf_ctx* c, const float* U, const float* v, float* Jv) {
  if (!c) return PF_ERR_ARG;
  pf_status st = check_ready(c);
  if (st != PF_OK) return st;
  if (!has_implicit(c)) return fail(c, PF_ERR_ARG, "pf_jvp supports 3-D meshes and 2-D AC / CH");
  if (!U || !v || !Jv) return fail(c, PF_ERR_ARG, "null array");
  PF_CUDA(jvp3d(c, U, v, Jv, 1));
  return PF_OK;
}

pf_status pf_implicit_residual(pf_ctx* c, const float* Un, const float* U, float* R) {
  if (!c) return PF_ERR_ARG;
  pf_status st = check_ready(c);
  if (st != PF_OK) return st;
  if (!has_implicit(c))
    return fail(c, PF_ERR_ARG, "pf_implicit_residual supports 3-D meshes and 2-D AC / CH");
  if (!U || !Un || !R) return fail(c, PF_ERR_ARG, "null array");
  PF_CUDA(residual3d(c, U, Un, R, 1));
  return PF_OK;
}

const char* pf_last_error(const pf_ctx* c) { return c ? c->err.c_str() : "null context"; }

void pf_destroy(pf_ctx* c) {
  if (!c) return;
  destroy_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

pf_status pf_implicit_adjoint_workspace(pf_ctx* c, int64_t n_steps, size_t* bytes) {
  if (!c || !bytes) return PF_ERR_ARG;
  if (!iadj_ok(c))
    return fail(c, PF_ERR_ARG, "the implicit adjoint needs a gradient-flow mesh (3-D, 2-D AC)");
  if (n_steps < 1) return fail(c, PF_ERR_ARG, "n_steps must be >= 1");
  *bytes = iadj_vec(c) * (size_t)(n_steps + 3) + 256;
  return PF_OK;
}

pf_status pf_implicit_adjoint(pf_ctx* c, const float* U0, int64_t n_steps,
                              const pf_newton_opts* opts, void* ws, size_t bytes,
                              double* objective, double* grads, pf_newton_stats* stats) {
  if (!c) return PF_ERR_ARG;
  pf_status st = check_ready(c);
  if (st != PF_OK) return st;
  size_t need = 0;
  if ((st = pf_implicit_adjoint_workspace(c, n_steps, &need)) != PF_OK) return st;
  if ((st = need_implicit_ws(c)) != PF_OK) return st;
  if (!U0 || !ws || !objective || !grads) return fail(c, PF_ERR_ARG, "null argument");
  if (bytes < need || (uintptr_t)ws % 256)
    return fail(c, PF_ERR_ARG, "implicit adjoint workspace too small or misaligned (%zu < %zu)",
                bytes, need);
  const int64_t n = vec_len(c);
  const size_t vb = iadj_vec(c);
  char* w = (char*)ws;
  auto traj = [&](int64_t s) { return (float*)(w + vb * (size_t)s); };
  float* lam = (float*)(w + vb * (size_t)(n_steps + 1));
  float* tmp = (float*)(w + vb * (size_t)(n_steps + 2));
  double* dscr = (double*)(w + vb * (size_t)(n_steps + 3));
  const int nz = c->dim == 3 ? (int)c->n[2] : 1;
  const double cell = c->h[0] * c->h[1] * c->h[2];
  const double dt = c->par.dt, L = c->par.mobility;
  pf_newton_stats tot{0, 0, 1, 0.0, 0.0};

  // forward: the implicit trajectory, every state kept
  PF_CUDA(cudaMemcpyAsync(traj(0), U0, sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream));
  for (int64_t s = 0; s < n_steps; ++s) {
    PF_CUDA(cudaMemcpyAsync(traj(s + 1), traj(s), sizeof(float) * n, cudaMemcpyDeviceToDevice,
                            c->stream));
    pf_newton_stats one{};
    st = pf_step_implicit(c, traj(s + 1), 1, nullptr, opts, &one);
    tot.newton_iters += one.newton_iters;
    tot.gmres_iters += one.gmres_iters;
    if (s == 0) tot.initial_residual = one.initial_residual;
    tot.final_residual = one.final_residual;
    if (st != PF_OK) {
      if (stats) *stats = tot;
      return st;
    }
  }
  // objective O = (1/V) sum_i m_i U^N_i (Eq. 19) and lambda^N = dO/dU^N = m / V
  double V = 1.0;
  for (int k = 0; k < c->dim; ++k) V *= (double)(c->n[k] - 1) * c->h[k];
  PF_CUDA(cudaMemsetAsync(tmp, 0, sizeof(float) * n, c->stream));
  PF_CUDA(pf::launch_add(tmp, tmp, n, 1.0f, c->stream));
  PF_CUDA(pf::launch_mass_mul(tmp, lam, (int)c->n[0], (int)c->n[1], nz, imp_nf(c), cell,
                              (float)(1.0 / V), 0, c->stream));
  if ((st = dot_host(c, lam, traj(n_steps), dscr, objective)) != PF_OK) return st;
  // reverse sweep: J(U^{n+1})^T mu = lambda (J symmetric), gradients, lambda <- M mu / dt
  grads[0] = grads[1] = 0.0;
  const int restart = opts ? opts->gmres_restart : 30;
  const int maxit = opts ? opts->gmres_max_iters : 300;
  // adjoint solves: relative tolerance 1e-6, or the caller's GMRES tolerance if tighter
  const double adj_rtol = (opts && opts->gmres_rtol > 0.0 && opts->gmres_rtol < 1e-6)
                              ? opts->gmres_rtol : 1e-6;
  for (int64_t s = n_steps - 1; s >= 0; --s) {
    const float* U = traj(s + 1);
    PF_CUDA(cudaMemcpyAsync(c->u, U, sizeof(float) * n, cudaMemcpyDeviceToDevice, c->stream));
    PF_CUDA(pf::launch_mass_mul(lam, c->g, (int)c->n[0], (int)c->n[1], nz, imp_nf(c), cell,
                                -1.0f, 1, c->stream));  // G = -M^-1 lambda
    int gi = 0;
    double rel = 0.0;
    if ((st = gmres3d(c, restart, 10 * maxit, adj_rtol, 0.0, &gi, &rel)) != PF_OK) return st;
    tot.gmres_iters += gi;
    double d = 0.0;
    PF_CUDA(residual3d(c, U, U, tmp, 1));  // L r(U)
    if ((st = dot_host(c, c->d, tmp, dscr, &d)) != PF_OK) return st;
    grads[0] -= d / L;                     // dC/dL = r(U)
    PF_CUDA(stiff_only(c, U, tmp));        // L K U
    if ((st = dot_host(c, c->d, tmp, dscr, &d)) != PF_OK) return st;
    grads[1] -= d;                         // dC/dkappa = L K U
    PF_CUDA(pf::launch_mass_mul(c->d, lam, (int)c->n[0], (int)c->n[1], nz, imp_nf(c), cell,
                                (float)(1.0 / dt), 0, c->stream));
  }
  if (stats) *stats = tot;
  if (!std::isfinite(*objective) || !std::isfinite(grads[0]) || !std::isfinite(grads[1]))
    return fail(c, PF_ERR_NONFINITE, "non-finite adjoint result");
  return PF_OK;
}

}  // extern "C"
