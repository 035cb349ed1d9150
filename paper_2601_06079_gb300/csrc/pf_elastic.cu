// C ABI of the Eshelby-inclusion elasticity path (JAX-PF Eq. 3-4, eigenstrain
// of Supp. 3 Eq. III.1, objective and sensitivities of Eq. 21-22): the
// stiffness operator, the loads, conjugate gradients with device-resident
// scalars, and the adjoint sensitivities of a linear objective to E and nu.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "pf_internal.h"

namespace {

using pf::Elastic3DArgs;
using pf::ElasticLoadArgs;

constexpr int kCheckEvery = 8;  // CG iterations between convergence checks on the host

// Element stiffness of the uniform box element in closed form:
//   K[(a,i),(b,j)] = lam I_ij(a,b) + mu (delta_ij sum_k I_kk(a,b) + I_ji(a,b)),
//   I_ij(a,b) = int d_i N_a d_j N_b dV,
// each I a product of exact 1-D integrals over [0, 1] of the linear shape
// functions and their derivatives (the trilinear integrand factorises per axis):
//   int N N = 1/3 (same end) or 1/6;  int N' N' = +-1;  int N' N = +-1/2.
void element_stiffness(const double h[3], double lam, double mu, double K[24][24]) {
  auto mass1 = [](int p, int q) { return p == q ? 1.0 / 3.0 : 1.0 / 6.0; };
  auto stiff1 = [](int p, int q) { return p == q ? 1.0 : -1.0; };
  auto dn = [](int p) { return p ? 1.0 : -1.0; };  // N_p' on [0, 1]
  const double vol = h[0] * h[1] * h[2];
  double I[8][8][3][3];
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b) {
      const int pa[3] = {a & 1, (a >> 1) & 1, a >> 2}, pb[3] = {b & 1, (b >> 1) & 1, b >> 2};
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          double v = vol / (h[i] * h[j]);
          for (int k = 0; k < 3; ++k) {
            if (k == i && k == j)
              v *= stiff1(pa[k], pb[k]);
            else if (k == i)
              v *= 0.5 * dn(pa[k]);  // int N_a' N_b
            else if (k == j)
              v *= 0.5 * dn(pb[k]);  // int N_a N_b'
            else
              v *= mass1(pa[k], pb[k]);
          }
          I[a][b][i][j] = v;
        }
    }
  for (int a = 0; a < 8; ++a)
    for (int b = 0; b < 8; ++b)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const double tr = I[a][b][0][0] + I[a][b][1][1] + I[a][b][2][2];
          K[a * 3 + i][b * 3 + j] = lam * I[a][b][i][j] + mu * ((i == j) * tr + I[a][b][j][i]);
        }
}

bool valid(const pf_elastic* e) {
  if (!e) return false;
  for (int k = 0; k < 3; ++k)
    if (e->n[k] < 2 || e->n[k] > (1 << 20) || !(e->h[k] > 0.0) || !isfinite(e->h[k])) return false;
  if ((double)e->n[0] * e->n[1] * e->n[2] * 3 > 4e9) return false;
  if (!(e->E > 0.0) || !isfinite(e->E) || !(e->nu > -1.0 && e->nu < 0.5)) return false;
  return isfinite(e->m) && isfinite(e->l) && isfinite(e->a);
}

int64_t nodes(const pf_elastic* e) { return e->n[0] * e->n[1] * e->n[2]; }

void lame(double E, double nu, double* lam, double* mu) {
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *mu = E / (2.0 * (1.0 + nu));
}

// derivatives of (lam, mu) with respect to E (k = 0) and nu (k = 1)
void dlame(double E, double nu, int k, double* dl, double* dm) {
  const double D = (1.0 + nu) * (1.0 - 2.0 * nu);
  if (k == 0) {
    *dl = nu / D;
    *dm = 1.0 / (2.0 * (1.0 + nu));
  } else {
    *dl = E * (1.0 + 2.0 * nu * nu) / (D * D);
    *dm = -E / (2.0 * (1.0 + nu) * (1.0 + nu));
  }
}

void fill_apply(const pf_elastic* e, double lam, double mu, int constrain, Elastic3DArgs* a) {
  double K[24][24];
  element_stiffness(e->h, lam, mu, K);
  a->nx = (int)e->n[0];
  a->ny = (int)e->n[1];
  a->nz = (int)e->n[2];
  a->constrain = constrain;
  a->dot = nullptr;
  for (int r = 0; r < 24; ++r)
    for (int c = 0; c < 24; ++c) a->ke[r * 24 + c] = (float)K[r][c];
  // assembled interior stencil: offset o = b - a over all 8 elements of a node
  double ks[27][3][3];
  memset(ks, 0, sizeof(ks));
  for (int an = 0; an < 8; ++an)
    for (int b = 0; b < 8; ++b) {
      const int o = ((b >> 2) - (an >> 2) + 1) * 9 + (((b >> 1) & 1) - ((an >> 1) & 1) + 1) * 3 +
                    ((b & 1) - (an & 1) + 1);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) ks[o][i][j] += K[an * 3 + i][b * 3 + j];
    }
  for (int o = 0; o < 27; ++o)
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) a->ks[(o * 3 + i) * 3 + j] = (float)ks[o][i][j];
}

void fill_load(const pf_elastic* e, int unit, double scale, int constrain, ElasticLoadArgs* a) {
  a->nx = (int)e->n[0];
  a->ny = (int)e->n[1];
  a->nz = (int)e->n[2];
  a->unit = unit;
  a->constrain = constrain;
  a->hx = (float)e->h[0];
  a->hy = (float)e->h[1];
  a->hz = (float)e->h[2];
  a->ihx = (float)(1.0 / e->h[0]);
  a->ihy = (float)(1.0 / e->h[1]);
  a->ihz = (float)(1.0 / e->h[2]);
  a->wq = (float)(e->h[0] * e->h[1] * e->h[2] / 8.0);
  a->scale = (float)scale;
  a->l = (float)e->l;
  a->a = (float)e->a;
}

// workspace: 7 vectors of 3N floats, then FP64 partials, 32 FP64 scalars and
// the block counter of the single-launch reductions
struct Layout {
  size_t vec, off_part, off_sc, total;
};
Layout layout(const pf_elastic* e) {
  Layout L;
  L.vec = ((size_t)(3 * nodes(e)) * sizeof(float) + 255) / 256 * 256;
  L.off_part = 7 * L.vec;
  // FP64 partials, shared in turn by the apply, the update and launch_dots
  size_t np = (size_t)pf::krylov_partial_blocks();
  np = std::max(np, (size_t)pf::cg_blocks());
  np = std::max(np, (size_t)pf::elastic_apply_blocks((int)e->n[0], (int)e->n[1], (int)e->n[2]));
  L.off_sc = L.off_part + (np * sizeof(double) + 255) / 256 * 256;
  L.total = L.off_sc + 512;
  return L;
}

#define EL_CUDA(x)                                  \
  do {                                              \
    if ((x) != cudaSuccess) return PF_ERR_CUDA;     \
  } while (0)

// One CG iteration (slot = iteration parity): Ap = K p with the p.Ap partials,
// sc[2] = p.Ap, x += alpha p, r -= alpha Ap with the new r.r partials,
// sc[1 - slot] = r.r, p = r + beta p.
cudaError_t cg_iteration(const Elastic3DArgs& A, int64_t n, int napply, float* x, float* r,
                         float* p, float* Ap, double* part, double* sc, int slot,
                         cudaStream_t s) {
  cudaError_t e;
  if ((e = pf::launch_elastic_apply(A, s)) != cudaSuccess) return e;
  if ((e = pf::launch_sum_part(part, napply, sc + 2, s)) != cudaSuccess) return e;
  if ((e = pf::launch_cg_xr(x, r, p, Ap, n, sc, slot, part, s)) != cudaSuccess) return e;
  if ((e = pf::launch_sum_part(part, pf::cg_blocks(), sc + (1 - slot), s)) != cudaSuccess) return e;
  return pf::launch_cg_p(r, p, n, sc, slot, s);
}

// K x = b on the free degrees of freedom (b's constrained entries are
// ignored), from x = 0; vectors r, p, Ap are workspace.  Iterations run in
// groups of kCheckEvery replayed from a CUDA graph (captured once per call on
// a private stream), with a convergence check on the host after each group.
pf_status cg(const pf_elastic* e, const Elastic3DArgs& base, const float* b, float* x, float* r,
             float* p, float* Ap, double* part, double* sc, unsigned* cnt, double rtol,
             int max_iter, cudaStream_t s, pf_cg_stats* st) {
  const int64_t N = nodes(e), n = 3 * N;
  EL_CUDA(cudaMemsetAsync(x, 0, sizeof(float) * n, s));
  EL_CUDA(cudaMemcpyAsync(r, b, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  EL_CUDA(pf::launch_elastic_constrain(r, base.nx, base.ny, base.nz, s));
  EL_CUDA(cudaMemcpyAsync(p, r, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
  EL_CUDA(pf::launch_dots(r, 0, 1, r, n, part, sc, cnt, s));
  double h_sc[2] = {0.0, 0.0};
  EL_CUDA(cudaMemcpyAsync(h_sc, sc, sizeof(double), cudaMemcpyDeviceToHost, s));
  EL_CUDA(cudaStreamSynchronize(s));
  const double rr0 = h_sc[0];
  if (!isfinite(rr0)) return PF_ERR_NONFINITE;
  if (st) {
    st->iterations = 0;
    st->converged = 0;
    st->initial_residual = sqrt(rr0);
    st->final_residual = sqrt(rr0);
  }
  if (rr0 == 0.0) {
    if (st) st->converged = 1;
    return PF_OK;
  }
  const double stop = rtol * rtol * rr0;
  Elastic3DArgs A = base;
  A.u = p;
  A.out = Ap;
  A.dot = part;
  const int napply = pf::elastic_apply_blocks(A.nx, A.ny, A.nz);
  // the graph of kCheckEvery iterations (even, so slots repeat per group)
  cudaGraphExec_t exec = nullptr;
  if (max_iter >= kCheckEvery) {
    cudaStream_t cs = nullptr;
    EL_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    cudaError_t le = cudaSuccess;
    if (ce == cudaSuccess) {
      for (int k = 0; k < kCheckEvery && le == cudaSuccess; ++k)
        le = cg_iteration(A, n, napply, x, r, p, Ap, part, sc, k & 1, cs);
      cudaGraph_t g = nullptr;
      ce = cudaStreamEndCapture(cs, &g);
      if (ce == cudaSuccess && le == cudaSuccess) ce = cudaGraphInstantiate(&exec, g, 0);
      if (g) cudaGraphDestroy(g);
    }
    cudaStreamDestroy(cs);
    if (ce != cudaSuccess || le != cudaSuccess) {
      if (exec) cudaGraphExecDestroy(exec);
      return PF_ERR_CUDA;
    }
  }
  int it = 0;
  double rr = rr0;
  pf_status result = PF_ERR_NOT_CONVERGED;
  while (it < max_iter) {
    cudaError_t le;
    if (exec && max_iter - it >= kCheckEvery) {
      le = cudaGraphLaunch(exec, s);
      it += kCheckEvery;
    } else {
      le = cg_iteration(A, n, napply, x, r, p, Ap, part, sc, it & 1, s);
      ++it;
    }
    if (le != cudaSuccess) {
      result = PF_ERR_CUDA;
      break;
    }
    if (it % kCheckEvery == 0 || it == max_iter) {
      if (cudaMemcpyAsync(h_sc, sc, 2 * sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
          cudaStreamSynchronize(s) != cudaSuccess) {
        result = PF_ERR_CUDA;
        break;
      }
      rr = h_sc[it & 1];  // the slot the last iteration wrote
      if (!isfinite(rr)) {
        result = PF_ERR_NONFINITE;
        break;
      }
      if (rr <= stop) {
        result = PF_OK;
        break;
      }
    }
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (st) {
    st->iterations = it;
    st->converged = result == PF_OK;
    st->final_residual = sqrt(rr);
  }
  return result;
}

}  // namespace

extern "C" {

pf_status pf_elastic_workspace(const pf_elastic* e, size_t* bytes) {
  if (!valid(e) || !bytes) return PF_ERR_ARG;
  *bytes = layout(e).total;
  return PF_OK;
}

pf_status pf_elastic_apply(const pf_elastic* e, const float* u, float* Ku, int constrain,
                           void* stream) {
  if (!valid(e) || !u || !Ku || u == Ku) return PF_ERR_ARG;
  double lam, mu;
  lame(e->E, e->nu, &lam, &mu);
  Elastic3DArgs a;
  fill_apply(e, lam, mu, constrain ? 1 : 0, &a);
  a.u = u;
  a.out = Ku;
  EL_CUDA(pf::launch_elastic_apply(a, (cudaStream_t)stream));
  return PF_OK;
}

pf_status pf_elastic_load(const pf_elastic* e, int unit, float* f, void* stream) {
  if (!valid(e) || !f) return PF_ERR_ARG;
  double lam, mu;
  lame(e->E, e->nu, &lam, &mu);
  ElasticLoadArgs a;
  fill_load(e, unit ? 1 : 0, unit ? 1.0 : (3.0 * lam + 2.0 * mu) * e->m, 0, &a);
  EL_CUDA(pf::launch_elastic_load(a, f, (cudaStream_t)stream));
  return PF_OK;
}

pf_status pf_elastic_solve(const pf_elastic* e, const float* b, float* u, double rtol,
                           int max_iter, void* ws, size_t bytes, void* stream, pf_cg_stats* stats) {
  if (!valid(e) || !u || !ws || max_iter < 1 || !(rtol > 0.0) || (uintptr_t)ws % 256)
    return PF_ERR_ARG;
  const Layout L = layout(e);
  if (bytes < L.total) return PF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  char* w = (char*)ws;
  float *r = (float*)w, *p = (float*)(w + L.vec), *Ap = (float*)(w + 2 * L.vec),
        *f = (float*)(w + 3 * L.vec);
  double* part = (double*)(w + L.off_part);
  double* sc = (double*)(w + L.off_sc);
  unsigned* cnt = (unsigned*)(w + L.off_sc + 256);
  EL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
  double lam, mu;
  lame(e->E, e->nu, &lam, &mu);
  if (!b) {
    ElasticLoadArgs la;
    fill_load(e, 0, (3.0 * lam + 2.0 * mu) * e->m, 1, &la);
    EL_CUDA(pf::launch_elastic_load(la, f, s));
    b = f;
  }
  Elastic3DArgs a;
  fill_apply(e, lam, mu, 1, &a);
  return cg(e, a, b, u, r, p, Ap, part, sc, cnt, rtol, max_iter, s, stats);
}

pf_status pf_elastic_sensitivity(const pf_elastic* e, const float* g, float* u, double rtol,
                                 int max_iter, void* ws, size_t bytes, void* stream,
                                 double* objective, double* grads, pf_cg_stats* stats) {
  if (!valid(e) || !u || !ws || !objective || !grads || max_iter < 1 || !(rtol > 0.0) ||
      (uintptr_t)ws % 256)
    return PF_ERR_ARG;
  const Layout L = layout(e);
  if (bytes < L.total) return PF_ERR_ARG;
  cudaStream_t s = (cudaStream_t)stream;
  const int64_t n = 3 * nodes(e);
  char* w = (char*)ws;
  float *r = (float*)w, *p = (float*)(w + L.vec), *Ap = (float*)(w + 2 * L.vec),
        *f = (float*)(w + 3 * L.vec), *gv = (float*)(w + 4 * L.vec),
        *la = (float*)(w + 5 * L.vec), *t = (float*)(w + 6 * L.vec);
  double* part = (double*)(w + L.off_part);
  double* sc = (double*)(w + L.off_sc);
  unsigned* cnt = (unsigned*)(w + L.off_sc + 256);
  EL_CUDA(cudaMemsetAsync(cnt, 0, sizeof(unsigned), s));
  double lam, mu;
  lame(e->E, e->nu, &lam, &mu);
  Elastic3DArgs a;
  fill_apply(e, lam, mu, 1, &a);
  ElasticLoadArgs ld;
  fill_load(e, 0, (3.0 * lam + 2.0 * mu) * e->m, 1, &ld);
  EL_CUDA(pf::launch_elastic_load(ld, f, s));
  pf_cg_stats st_u = {}, st_l = {};
  pf_status rs = cg(e, a, f, u, r, p, Ap, part, sc, cnt, rtol, max_iter, s, &st_u);
  if (rs != PF_OK) {
    if (stats) *stats = st_u;
    return rs;
  }
  // objective functional: the caller's g, or the small-strain volume
  double V0 = 0.0;
  if (g) {
    EL_CUDA(cudaMemcpyAsync(gv, g, sizeof(float) * n, cudaMemcpyDeviceToDevice, s));
    EL_CUDA(pf::launch_elastic_constrain(gv, a.nx, a.ny, a.nz, s));
  } else {
    ElasticLoadArgs lv;
    fill_load(e, 1, 1.0, 1, &lv);
    EL_CUDA(pf::launch_elastic_load(lv, gv, s));
    V0 = (double)(e->n[0] - 1) * e->h[0] * (double)(e->n[1] - 1) * e->h[1] *
         (double)(e->n[2] - 1) * e->h[2];
  }
  double h_d[3];
  EL_CUDA(pf::launch_dots(gv, 0, 1, u, n, part, sc + 3, cnt, s));
  rs = cg(e, a, gv, la, r, p, Ap, part, sc, cnt, rtol, max_iter, s, &st_l);
  if (rs != PF_OK) {
    if (stats) *stats = st_l;
    return rs;
  }
  for (int k = 0; k < 2; ++k) {
    double dl, dm;
    dlame(e->E, e->nu, k, &dl, &dm);
    Elastic3DArgs ak;
    fill_apply(e, dl, dm, 1, &ak);
    ak.u = u;
    ak.out = t;
    EL_CUDA(pf::launch_elastic_apply(ak, s));
    ElasticLoadArgs lk;
    fill_load(e, 0, (3.0 * dl + 2.0 * dm) * e->m, 1, &lk);
    EL_CUDA(pf::launch_elastic_load(lk, Ap, s));
    EL_CUDA(pf::launch_axpby(1.0f, Ap, -1.0f, t, n, s));  // t = df - dK u
    EL_CUDA(pf::launch_dots(la, 0, 1, t, n, part, sc + 4 + k, cnt, s));
  }
  EL_CUDA(cudaMemcpyAsync(h_d, sc + 3, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
  EL_CUDA(cudaStreamSynchronize(s));
  *objective = V0 + h_d[0];
  grads[0] = h_d[1];
  grads[1] = h_d[2];
  if (stats) {
    *stats = st_u;
    stats->iterations += st_l.iterations;
  }
  if (!isfinite(*objective) || !isfinite(grads[0]) || !isfinite(grads[1])) return PF_ERR_NONFINITE;
  return PF_OK;
}

}  // extern "C"
