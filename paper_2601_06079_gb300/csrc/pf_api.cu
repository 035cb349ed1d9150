// C ABI of libpf: context, workspace carving, parameter derivation and the
// host-side drivers that enqueue the kernels.  No device memory is allocated
// here; all scratch lives in the caller's workspace.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <string>

#include "pf_internal.h"

struct pf_ctx {
  int dim = 2;
  int64_t n[3] = {1, 1, 1};
  double h[3] = {1, 1, 1};
  pf_model model = PF_MODEL_AC;
  int nf = 1;
  cudaStream_t stream = nullptr;

  size_t ws_bytes = 0;
  char* ws = nullptr;
  pf_params par{};
  bool par_set = false;

  // workspace segments
  float* buf_a = nullptr;
  float* buf_b = nullptr;
  double* partials = nullptr;
  double* result = nullptr;

  // derived coefficients
  pf::Explicit2DArgs ex{};

  // CUDA graph of kGraphSteps explicit steps buf_a -> ... -> buf_a
  cudaStream_t cap_stream = nullptr;
  cudaGraphExec_t graph = nullptr;

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

struct Layout {
  size_t a, b, partials, result, total;
};

Layout layout(const pf_ctx* c) {
  Layout L{};
  const size_t field =
      align_up(sizeof(float) * (size_t)pf::work_pitch((int)c->n[0]) * pf::work_rows((int)c->n[1]), 256);
  size_t off = 0;
  L.a = off;
  off += field;
  L.b = off;
  off += field;
  L.partials = off;
  off += align_up(sizeof(double) * 2 * 1024, 256);
  L.result = off;
  off += 256;
  L.total = off;
  return L;
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

void destroy_graph(pf_ctx* c) {
  if (c->graph) cudaGraphExecDestroy(c->graph);
  c->graph = nullptr;
}

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

}  // namespace

extern "C" {

pf_status pf_create_mesh(pf_ctx** out, int dim, const int64_t nodes[3], const double h[3],
                         pf_model model, int n_fields, void* stream, size_t* workspace_bytes) {
  if (!out || !nodes || !h || !workspace_bytes) return PF_ERR_ARG;
  *out = nullptr;
  if (dim != 2) return PF_ERR_ARG;  // 2-D explicit AC / CH
  if (model != PF_MODEL_AC && model != PF_MODEL_CH) return PF_ERR_ARG;
  if (n_fields != 1) return PF_ERR_ARG;
  const int64_t minn = (model == PF_MODEL_CH) ? 3 : 2;
  for (int k = 0; k < dim; ++k) {
    if (nodes[k] < minn || nodes[k] > (int64_t)1 << 20) return PF_ERR_ARG;
    if (!(h[k] > 0.0) || !isfinite(h[k])) return PF_ERR_ARG;
  }
  if (nodes[0] * nodes[1] > ((int64_t)1 << 31) - 1) return PF_ERR_ARG;
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
  c->ws_bytes = layout(c).total;
  *workspace_bytes = c->ws_bytes;
  *out = c;
  return PF_OK;
}

pf_status pf_bind_workspace(pf_ctx* c, void* dev_ptr, size_t bytes) {
  if (!c) return PF_ERR_ARG;
  if (!dev_ptr || (uintptr_t)dev_ptr % 256 != 0)
    return fail(c, PF_ERR_ARG, "workspace must be a non-null 256-byte aligned device pointer");
  if (bytes < c->ws_bytes)
    return fail(c, PF_ERR_ARG, "workspace too small: %zu < %zu bytes", bytes, c->ws_bytes);
  const Layout L = layout(c);
  c->ws = (char*)dev_ptr;
  c->buf_a = (float*)(c->ws + L.a);
  c->buf_b = (float*)(c->ws + L.b);
  c->partials = (double*)(c->ws + L.partials);
  c->result = (double*)(c->ws + L.result);
  destroy_graph(c);
  return PF_OK;
}

pf_status pf_set_params(pf_ctx* c, const pf_params* p) {
  if (!c) return PF_ERR_ARG;
  if (!p) return fail(c, PF_ERR_ARG, "params is NULL");
  if (!(p->dt > 0.0) || !(p->kappa >= 0.0) || !(p->mobility > 0.0) || !(p->W >= 0.0) ||
      !isfinite(p->dt) || !isfinite(p->kappa) || !isfinite(p->mobility) || !isfinite(p->W) ||
      !isfinite(p->shift))
    return fail(c, PF_ERR_ARG, "invalid parameters (need dt > 0, mobility > 0, kappa, W >= 0)");
  if (p->mobility_field)
    return fail(c, PF_ERR_ARG, "per-node mobility field is not supported by pf_step_explicit yet");
  c->par = *p;
  c->par_set = true;

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
  }
  pf::pack_explicit2d(a);
  destroy_graph(c);
  return PF_OK;
}

pf_status pf_step_explicit(pf_ctx* c, float* state, int64_t n_steps) {
  if (!c) return PF_ERR_ARG;
  if (!c->ws) return fail(c, PF_ERR_STATE, "no workspace bound");
  if (!c->par_set) return fail(c, PF_ERR_STATE, "parameters not set");
  if (!state) return fail(c, PF_ERR_ARG, "state is NULL");
  if (n_steps < 0) return fail(c, PF_ERR_ARG, "n_steps < 0");
  if (n_steps == 0) return PF_OK;
  const float shift = (float)c->par.shift;
  const int nx = (int)c->n[0], ny = (int)c->n[1];
  // working copies with the mirror frame: d = u - shift (both planes fully defined)
  PF_CUDA(pf::launch_to_work(state, c->buf_a, nx, ny, shift, c->stream));
  PF_CUDA(pf::launch_to_work(state, c->buf_b, nx, ny, shift, c->stream));
  int64_t left = n_steps;
  if (left >= kGraphSteps) {
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

const char* pf_last_error(const pf_ctx* c) { return c ? c->err.c_str() : "null context"; }

void pf_destroy(pf_ctx* c) {
  if (!c) return;
  destroy_graph(c);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
