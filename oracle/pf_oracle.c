/*
 * FP64 CPU oracle for the Q1 finite-element phase-field method.
 *
 * TEST INFRASTRUCTURE.  Only the tests, the package smoke check and the
 * bench's CPU-baseline leg may load this library.  It is a plain, slow,
 * element-by-element restatement of the paper's discretised equations and
 * shares nothing with the CUDA path.
 *
 * Every routine loops over elements and Gauss points exactly as the weak
 * form is written, with no blocking, no stencil shortcuts and no fused
 * passes.  OpenMP only splits the element loop into 2^dim colours (elements
 * of one colour share no node), which changes nothing but the order of the
 * additions into a node.
 *
 * Sources (JAX-PF, Hu et al.):
 *   Eq. 1, 2    Allen-Cahn and Cahn-Hilliard evolution laws
 *   Eq. 5, 6    free energy = local density + kappa/2 |grad u|^2
 *   Eq. 9, 10   split Cahn-Hilliard form with unknowns c and mu
 *   Eq. 11      semi-discrete system M dU/dt + r(U, theta) = 0
 *   Eq. 12      explicit Euler update U <- U - dt M^-1 r(U)
 *   Eq. 13, 14  implicit Euler residual R = M (U - U^n)/dt + r(U)
 *   Supp. 2     adjoint sensitivities (here the discrete adjoint of Eq. 12)
 */
#include <omp.h>
#include "pf_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

#define MAXA 8

/* Reference element built from the definitions: Q1 shape functions
 * N_a(xi) = prod_k (xi_k or 1 - xi_k) on the unit cell, Gauss points at
 * (1 -+ 1/sqrt 3)/2 per axis with weight 1/2 each, mapped to an h-sized cell. */
typedef struct {
  int nn, nq;
  double N[MAXA][MAXA];     /* N[q][a] */
  double G[MAXA][MAXA][3];  /* d N_a / d x_k at point q */
  double wq;                /* weight times |J| of every Gauss point */
} or_elem;

static void ref_element(const or_mesh* m, or_elem* e) {
  const double gpt[2] = {0.5 * (1.0 - 1.0 / sqrt(3.0)), 0.5 * (1.0 + 1.0 / sqrt(3.0))};
  const int d = m->dim;
  e->nn = 1 << d;
  e->nq = 1 << d;
  double vol = 1.0;
  for (int k = 0; k < d; ++k) vol *= m->h[k];
  e->wq = vol / e->nq;
  for (int q = 0; q < e->nq; ++q) {
    double xi[3];
    for (int k = 0; k < d; ++k) xi[k] = gpt[(q >> k) & 1];
    for (int a = 0; a < e->nn; ++a) {
      double val = 1.0;
      for (int k = 0; k < d; ++k) val *= ((a >> k) & 1) ? xi[k] : 1.0 - xi[k];
      e->N[q][a] = val;
      for (int k = 0; k < 3; ++k) e->G[q][a][k] = 0.0;
      for (int k = 0; k < d; ++k) {
        double g = (((a >> k) & 1) ? 1.0 : -1.0) / m->h[k];
        for (int l = 0; l < d; ++l)
          if (l != k) g *= ((a >> l) & 1) ? xi[l] : 1.0 - xi[l];
        e->G[q][a][k] = g;
      }
    }
  }
}

int64_t or_nnodes(const or_mesh* m) {
  return m->n[0] * m->n[1] * (m->dim == 3 ? m->n[2] : 1);
}

/* ---- local free-energy density and its derivatives (Eq. 5-7) ---------- */

/* Coupled Allen-Cahn / Cahn-Hilliard (Eq. 7) with the polynomials printed in
 * Supp. 3: phase free energies f_alpha(c), f_beta(c) and the interpolation
 * h(eta) = 10 eta^3 - 15 eta^4 + 6 eta^5.  Coefficients in increasing powers. */
static const double kFa[5] = {-1.6704, -4.776, 5.1622, -2.7375, 1.3687};
static const double kFb[3] = {-1.5924, -5.9746, 5.0};

static double poly(const double* a, int n, double x) {
  double s = 0.0;
  for (int k = n - 1; k >= 0; --k) s = s * x + a[k];
  return s;
}
static double dpoly(const double* a, int n, double x) {
  double s = 0.0;
  for (int k = n - 1; k >= 1; --k) s = s * x + k * a[k];
  return s;
}
static double d2poly(const double* a, int n, double x) {
  double s = 0.0;
  for (int k = n - 1; k >= 2; --k) s = s * x + k * (k - 1) * a[k];
  return s;
}
static const double kH[6] = {0.0, 0.0, 0.0, 10.0, -15.0, 6.0};

/* gradient-energy coefficient of field f: the coupled model has no c gradient term */
static double kappa_of(const or_params* p, int f) {
  return (p->energy == OR_COUPLED && f == 0) ? 0.0 : p->kappa;
}

static double f_local(const or_params* p, const double* u) {
  if (p->energy == OR_COUPLED) {
    const double h = poly(kH, 6, u[1]);
    return poly(kFa, 5, u[0]) * (1.0 - h) + poly(kFb, 3, u[0]) * h;
  }
  if (p->energy == OR_DOUBLE_WELL) {
    double c = u[0];
    return p->W * c * c * (1.0 - c) * (1.0 - c);
  }
  double s = 0.0;
  for (int i = 0; i < p->nf; ++i) {
    double e2 = u[i] * u[i];
    s += -0.5 * p->alpha * e2 + 0.25 * p->beta * e2 * e2;
    for (int j = i + 1; j < p->nf; ++j) s += p->gamma * e2 * u[j] * u[j];
  }
  return s;
}

static void df_local(const or_params* p, const double* u, double* g) {
  if (p->energy == OR_COUPLED) {
    const double h = poly(kH, 6, u[1]);
    g[0] = dpoly(kFa, 5, u[0]) * (1.0 - h) + dpoly(kFb, 3, u[0]) * h;
    g[1] = (poly(kFb, 3, u[0]) - poly(kFa, 5, u[0])) * dpoly(kH, 6, u[1]);
    return;
  }
  if (p->energy == OR_DOUBLE_WELL) {
    double c = u[0];
    g[0] = 2.0 * p->W * c * (1.0 - c) * (1.0 - 2.0 * c);
    return;
  }
  for (int i = 0; i < p->nf; ++i) {
    double others = 0.0;
    for (int j = 0; j < p->nf; ++j)
      if (j != i) others += u[j] * u[j];
    g[i] = -p->alpha * u[i] + p->beta * u[i] * u[i] * u[i] + 2.0 * p->gamma * u[i] * others;
  }
}

static void d2f_local(const or_params* p, const double* u, double* H) {
  const int nf = p->nf;
  if (p->energy == OR_COUPLED) {
    const double h = poly(kH, 6, u[1]), dh = dpoly(kH, 6, u[1]);
    H[0] = d2poly(kFa, 5, u[0]) * (1.0 - h) + d2poly(kFb, 3, u[0]) * h;
    H[1] = H[2] = (dpoly(kFb, 3, u[0]) - dpoly(kFa, 5, u[0])) * dh;
    H[3] = (poly(kFb, 3, u[0]) - poly(kFa, 5, u[0])) * d2poly(kH, 6, u[1]);
    return;
  }
  if (p->energy == OR_DOUBLE_WELL) {
    double c = u[0];
    H[0] = 2.0 * p->W * (1.0 - 6.0 * c + 6.0 * c * c);
    return;
  }
  for (int i = 0; i < nf; ++i) {
    double others = 0.0;
    for (int j = 0; j < nf; ++j)
      if (j != i) others += u[j] * u[j];
    for (int j = 0; j < nf; ++j)
      H[i * nf + j] = (i == j) ? (-p->alpha + 3.0 * p->beta * u[i] * u[i] + 2.0 * p->gamma * others)
                               : 4.0 * p->gamma * u[i] * u[j];
  }
}

/* ---- element loop ------------------------------------------------------ */

typedef void (*elem_fn)(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* ctx);

static void for_each_element(const or_mesh* m, const or_elem* e, elem_fn fn, void* ctx) {
  const int d = m->dim;
  const int64_t ne0 = m->n[0] - 1, ne1 = m->n[1] - 1, ne2 = (d == 3) ? m->n[2] - 1 : 1;
  const int64_t n0 = m->n[0], n1 = m->n[1];
  for (int col = 0; col < (1 << d); ++col) {
    const int64_t o0 = col & 1, o1 = (col >> 1) & 1, o2 = (col >> 2) & 1;
    const int64_t c0 = (ne0 - o0 + 1) / 2, c1 = (ne1 - o1 + 1) / 2, c2 = (ne2 - o2 + 1) / 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t kk = 0; kk < c2; ++kk)
      for (int64_t jj = 0; jj < c1; ++jj)
        for (int64_t ii = 0; ii < c0; ++ii) {
          const int64_t ei = 2 * ii + o0, ej = 2 * jj + o1, ek = 2 * kk + o2;
          int64_t nodes[MAXA];
          for (int a = 0; a < e->nn; ++a)
            nodes[a] = ((ek + ((a >> 2) & 1)) * n1 + (ej + ((a >> 1) & 1))) * n0 + (ei + (a & 1));
          fn(m, e, nodes, ctx);
        }
  }
}

/* values and gradients of field f at Gauss point q */
static void interp(const or_elem* e, const int64_t* nodes, const double* F, int q,
                   double* val, double* grad) {
  double v = 0.0, g0 = 0.0, g1 = 0.0, g2 = 0.0;
  for (int a = 0; a < e->nn; ++a) {
    const double ua = F[nodes[a]];
    v += e->N[q][a] * ua;
    g0 += e->G[q][a][0] * ua;
    g1 += e->G[q][a][1] * ua;
    g2 += e->G[q][a][2] * ua;
  }
  *val = v;
  grad[0] = g0;
  grad[1] = g1;
  grad[2] = g2;
}

/* ---- lumped mass: m_i = sum_e sum_q w |J| N_i(q) (row sum of Eq. 11's M) */

typedef struct { double* mass; } mass_ctx;

static void mass_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  (void)m;
  mass_ctx* c = (mass_ctx*)vctx;
  for (int a = 0; a < e->nn; ++a) {
    double s = 0.0;
    for (int q = 0; q < e->nq; ++q) s += e->wq * e->N[q][a];
    c->mass[nodes[a]] += s;
  }
}

void or_lumped_mass(const or_mesh* m, double* mass) {
  or_elem e;
  ref_element(m, &e);
  memset(mass, 0, sizeof(double) * or_nnodes(m));
  mass_ctx c = {mass};
  for_each_element(m, &e, mass_elem, &c);
}

/* ---- discrete energy E_h = sum_e sum_q w|J| [f(u_q) + kappa/2 |grad u_q|^2] (Eq. 5-6) */

typedef struct { const or_params* p; const double* U; int64_t NN; double* per_elem; } energy_ctx;

static void energy_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  energy_ctx* c = (energy_ctx*)vctx;
  const int nf = c->p->nf;
  double s = 0.0;
  for (int q = 0; q < e->nq; ++q) {
    double u[MAXA], grad2 = 0.0;
    for (int f = 0; f < nf; ++f) {
      double g[3];
      interp(e, nodes, c->U + f * c->NN, q, &u[f], g);
      grad2 += kappa_of(c->p, f) * (g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    }
    s += e->wq * (f_local(c->p, u) + 0.5 * grad2);
  }
  /* the element's first node identifies it uniquely */
  c->per_elem[nodes[0]] = s;
  (void)m;
}

double or_energy(const or_mesh* m, const or_params* p, const double* U) {
  or_elem e;
  ref_element(m, &e);
  const int64_t NN = or_nnodes(m);
  double* per = (double*)calloc(NN, sizeof(double));
  energy_ctx c = {p, U, NN, per};
  for_each_element(m, &e, energy_elem, &c);
  double s = 0.0;
  for (int64_t i = 0; i < NN; ++i) s += per[i];
  free(per);
  return s;
}

/* ---- residual r_i = dE_h/dU_i: sum_e sum_q w|J| [f'(u_q) N_i + kappa grad u_q . grad N_i] */

typedef struct { const or_params* p; const double* U; double* r; int64_t NN; } res_ctx;

static void residual_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  res_ctx* c = (res_ctx*)vctx;
  const int nf = c->p->nf;
  for (int q = 0; q < e->nq; ++q) {
    double u[MAXA], g[MAXA][3], df[MAXA];
    for (int f = 0; f < nf; ++f) interp(e, nodes, c->U + f * c->NN, q, &u[f], g[f]);
    df_local(c->p, u, df);
    for (int f = 0; f < nf; ++f)
      for (int a = 0; a < e->nn; ++a) {
        double gradterm = 0.0;
        for (int k = 0; k < m->dim; ++k) gradterm += g[f][k] * e->G[q][a][k];
        c->r[f * c->NN + nodes[a]] += e->wq * (df[f] * e->N[q][a] + kappa_of(c->p, f) * gradterm);
      }
  }
}

void or_residual(const or_mesh* m, const or_params* p, const double* U, double* r) {
  or_elem e;
  ref_element(m, &e);
  const int64_t NN = or_nnodes(m);
  memset(r, 0, sizeof(double) * NN * p->nf);
  res_ctx c = {p, U, r, NN};
  for_each_element(m, &e, residual_elem, &c);
}

/* ---- Hessian of E_h applied to v: sum_e sum_q w|J| [f''(u_q) v_q N_i + kappa grad v_q . grad N_i] */

typedef struct { const or_params* p; const double* U; const double* v; double* out; int64_t NN; } hess_ctx;

static void hessian_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  hess_ctx* c = (hess_ctx*)vctx;
  const int nf = c->p->nf;
  for (int q = 0; q < e->nq; ++q) {
    double u[MAXA], gu[3], vq[MAXA], gv[MAXA][3], H[MAXA * MAXA];
    for (int f = 0; f < nf; ++f) {
      interp(e, nodes, c->U + f * c->NN, q, &u[f], gu);
      interp(e, nodes, c->v + f * c->NN, q, &vq[f], gv[f]);
    }
    d2f_local(c->p, u, H);
    for (int f = 0; f < nf; ++f) {
      double hv = 0.0;
      for (int g2 = 0; g2 < nf; ++g2) hv += H[f * nf + g2] * vq[g2];
      for (int a = 0; a < e->nn; ++a) {
        double gradterm = 0.0;
        for (int k = 0; k < m->dim; ++k) gradterm += gv[f][k] * e->G[q][a][k];
        c->out[f * c->NN + nodes[a]] += e->wq * (hv * e->N[q][a] + kappa_of(c->p, f) * gradterm);
      }
    }
  }
}

void or_hessian_apply(const or_mesh* m, const or_params* p, const double* U, const double* v,
                      double* out) {
  or_elem e;
  ref_element(m, &e);
  const int64_t NN = or_nnodes(m);
  memset(out, 0, sizeof(double) * NN * p->nf);
  hess_ctx c = {p, U, v, out, NN};
  for_each_element(m, &e, hessian_elem, &c);
}

/* ---- mobility-weighted stiffness: (K_M mu)_i = sum_e sum_q w|J| M_q grad mu_q . grad N_i
 * with M_q = M * sum_b N_b(q) m_b (per-node multiplier m interpolated by Q1), Eq. 9 */

typedef struct { const or_params* p; const double* mu; double* out; } mob_ctx;

static double mobility_at(const or_params* p, const or_elem* e, const int64_t* nodes, int q) {
  double mq = 1.0;
  if (p->mob_field) {
    mq = 0.0;
    for (int b = 0; b < e->nn; ++b) mq += e->N[q][b] * p->mob_field[nodes[b]];
  }
  return p->mob * mq;
}

static void mobstiff_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  mob_ctx* c = (mob_ctx*)vctx;
  for (int q = 0; q < e->nq; ++q) {
    double v, g[3];
    interp(e, nodes, c->mu, q, &v, g);
    const double Mq = mobility_at(c->p, e, nodes, q);
    for (int a = 0; a < e->nn; ++a) {
      double gradterm = 0.0;
      for (int k = 0; k < m->dim; ++k) gradterm += g[k] * e->G[q][a][k];
      c->out[nodes[a]] += e->wq * Mq * gradterm;
    }
  }
}

void or_mobility_stiffness_apply(const or_mesh* m, const or_params* p, const double* mu,
                                 double* out) {
  or_elem e;
  ref_element(m, &e);
  memset(out, 0, sizeof(double) * or_nnodes(m));
  mob_ctx c = {p, mu, out};
  for_each_element(m, &e, mobstiff_elem, &c);
}

/* ---- explicit Euler, Eq. 12 with the lumped mass ----------------------- */

/* Allen-Cahn: M dU/dt = -L r(U)  =>  U <- U - dt L r(U) / m */
void or_ac_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps, double* U) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  double* r = (double*)malloc(sizeof(double) * NN * p->nf);
  or_lumped_mass(m, mass);
  for (int64_t s = 0; s < nsteps; ++s) {
    or_residual(m, p, U, r);
    for (int f = 0; f < p->nf; ++f)
      for (int64_t i = 0; i < NN; ++i) U[f * NN + i] -= dt * p->mob * r[f * NN + i] / mass[i];
  }
  free(r);
  free(mass);
}

/* Split Cahn-Hilliard (Eq. 9-10, read as mu = f'(c) - kappa lap c):
 * m_i mu_i = r_i(c) (the Allen-Cahn residual of c), then
 * m dc/dt = -K_M mu  =>  c <- c - dt K_M mu / m */
void or_ch_chemical_potential(const or_mesh* m, const or_params* p, const double* c, double* mu) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  or_residual(m, p, c, mu);
  for (int64_t i = 0; i < NN; ++i) mu[i] /= mass[i];
  free(mass);
}

void or_ch_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps, double* c) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  double* mu = (double*)malloc(sizeof(double) * NN);
  double* kmu = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  for (int64_t s = 0; s < nsteps; ++s) {
    or_residual(m, p, c, mu);
    for (int64_t i = 0; i < NN; ++i) mu[i] /= mass[i];
    or_mobility_stiffness_apply(m, p, mu, kmu);
    for (int64_t i = 0; i < NN; ++i) c[i] -= dt * kmu[i] / mass[i];
  }
  free(kmu);
  free(mu);
  free(mass);
}

/* Coupled Allen-Cahn / Cahn-Hilliard, explicit Euler with the lumped mass
 * (Eq. 1-2 and 9-12 with the energy of Eq. 7):
 *   m_i mu_i = dE_h/dc_i,  c <- c - dt K_{M_c} mu / m        (conserved c)
 *   eta <- eta - dt M_eta (dE_h/deta) / m                     (non-conserved eta)
 * both from the state at the start of the step. */
void or_coupled_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                         double* U) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  double* r = (double*)malloc(sizeof(double) * NN * 2);
  double* kmu = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  for (int64_t s = 0; s < nsteps; ++s) {
    or_residual(m, p, U, r);
    for (int64_t i = 0; i < NN; ++i) r[i] /= mass[i];       /* mu */
    or_mobility_stiffness_apply(m, p, r, kmu);                /* K_{M_c} mu (p->mob = M_c) */
    for (int64_t i = 0; i < NN; ++i) {
      U[i] -= dt * kmu[i] / mass[i];
      U[NN + i] -= dt * p->mob2 * r[NN + i] / mass[i];
    }
  }
  free(kmu);
  free(r);
  free(mass);
}

double or_mass_integral(const or_mesh* m, const double* c) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  double s = 0.0;
  for (int64_t i = 0; i < NN; ++i) s += mass[i] * c[i];
  free(mass);
  return s;
}

/* ---- implicit Euler, Eq. 13-14: R(U) = M (U - U^n)/dt + L r(U) --------- */

void or_implicit_residual(const or_mesh* m, const or_params* p, double dt, const double* Un,
                          const double* U, double* R) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  or_residual(m, p, U, R);
  for (int f = 0; f < p->nf; ++f)
    for (int64_t i = 0; i < NN; ++i) {
      const int64_t k = f * NN + i;
      R[k] = mass[i] * (U[k] - Un[k]) / dt + p->mob * R[k];
    }
  free(mass);
}

/* dR/dU applied to v: M v / dt + L * Hessian(U) v */
void or_implicit_jvp(const or_mesh* m, const or_params* p, double dt, const double* U,
                     const double* v, double* Jv) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  or_hessian_apply(m, p, U, v, Jv);
  for (int f = 0; f < p->nf; ++f)
    for (int64_t i = 0; i < NN; ++i) {
      const int64_t k = f * NN + i;
      Jv[k] = mass[i] * v[k] / dt + p->mob * Jv[k];
    }
  free(mass);
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Textbook restarted GMRES(restart) (Saad & Schultz 1986) for J x = b with
 * modified Gram-Schmidt and Givens rotations; J is applied by `apply`, x holds
 * the initial guess.  Returns 1 when ||b - J x|| <= rtol ||b||. */
typedef void (*or_apply_fn)(const void* ctx, const double* x, double* y);

static int gmres_op(or_apply_fn apply, const void* ctx, int64_t n, const double* b, double* x,
                    int restart, int maxit, double rtol, int* iters_out) {
  const int R = restart;
  double* V = (double*)malloc(sizeof(double) * n * (R + 1));
  double* H = (double*)calloc((size_t)(R + 1) * R, sizeof(double));
  double* cs = (double*)malloc(sizeof(double) * R);
  double* sn = (double*)malloc(sizeof(double) * R);
  double* g = (double*)malloc(sizeof(double) * (R + 1));
  double* y = (double*)malloc(sizeof(double) * R);
  double* w = (double*)malloc(sizeof(double) * n);
  const double bnorm = sqrt(dot(b, b, n));
  int total = 0, converged = 0;
  if (bnorm == 0.0) {
    memset(x, 0, sizeof(double) * n);
    converged = 1;
  }
  while (!converged && total < maxit) {
    apply(ctx, x, w);
    for (int64_t i = 0; i < n; ++i) V[i] = b[i] - w[i];
    double beta = sqrt(dot(V, V, n));
    if (beta <= rtol * bnorm) { converged = 1; break; }
    for (int64_t i = 0; i < n; ++i) V[i] /= beta;
    memset(g, 0, sizeof(double) * (R + 1));
    g[0] = beta;
    int k = 0;
    for (; k < R && total < maxit; ++k, ++total) {
      double* vk1 = V + (int64_t)(k + 1) * n;
      apply(ctx, V + (int64_t)k * n, vk1);
      for (int j = 0; j <= k; ++j) {
        const double hjk = dot(vk1, V + (int64_t)j * n, n);
        H[j * R + k] = hjk;
        for (int64_t i = 0; i < n; ++i) vk1[i] -= hjk * V[(int64_t)j * n + i];
      }
      const double hk1 = sqrt(dot(vk1, vk1, n));
      H[(k + 1) * R + k] = hk1;
      if (hk1 > 0.0)
        for (int64_t i = 0; i < n; ++i) vk1[i] /= hk1;
      for (int j = 0; j < k; ++j) {
        const double t = cs[j] * H[j * R + k] + sn[j] * H[(j + 1) * R + k];
        H[(j + 1) * R + k] = -sn[j] * H[j * R + k] + cs[j] * H[(j + 1) * R + k];
        H[j * R + k] = t;
      }
      const double den = hypot(H[k * R + k], H[(k + 1) * R + k]);
      cs[k] = H[k * R + k] / den;
      sn[k] = H[(k + 1) * R + k] / den;
      H[k * R + k] = den;
      H[(k + 1) * R + k] = 0.0;
      g[k + 1] = -sn[k] * g[k];
      g[k] = cs[k] * g[k];
      if (fabs(g[k + 1]) <= rtol * bnorm) { ++k; ++total; converged = 1; break; }
    }
    for (int i = k - 1; i >= 0; --i) {
      double s = g[i];
      for (int j = i + 1; j < k; ++j) s -= H[i * R + j] * y[j];
      y[i] = s / H[i * R + i];
    }
    for (int j = 0; j < k; ++j)
      for (int64_t i = 0; i < n; ++i) x[i] += y[j] * V[(int64_t)j * n + i];
  }
  if (iters_out) *iters_out = total;
  free(V); free(H); free(cs); free(sn); free(g); free(y); free(w);
  return converged;
}

typedef struct { const or_mesh* m; const or_params* p; double dt; const double* U; } jvp_ctx;

static void apply_implicit_jvp(const void* vctx, const double* x, double* y) {
  const jvp_ctx* c = (const jvp_ctx*)vctx;
  or_implicit_jvp(c->m, c->p, c->dt, c->U, x, y);
}

int or_gmres(const or_mesh* m, const or_params* p, double dt, const double* U, const double* b,
             double* x, int restart, int maxit, double rtol, int* iters_out) {
  const jvp_ctx ctx = {m, p, dt, U};
  return gmres_op(apply_implicit_jvp, &ctx, or_nnodes(m) * p->nf, b, x, restart, maxit, rtol,
                  iters_out);
}

/* Newton-Raphson on a residual R(U) with Jacobian action J (U holds the initial
 * guess on entry, the root on exit); each correction solves J d = -R with
 * GMRES.  Returns 1 when ||R||_2 <= abs_tol. */
typedef void (*or_residual_fn)(const void* ctx, const double* U, double* R);
typedef void (*or_jacobian_fn)(const void* ctx, const double* U, const double* v, double* Jv);

typedef struct { or_jacobian_fn jac; const void* ctx; const double* U; } lin_ctx;

static void apply_linearised(const void* vctx, const double* x, double* y) {
  const lin_ctx* c = (const lin_ctx*)vctx;
  c->jac(c->ctx, c->U, x, y);
}

static int newton_op(or_residual_fn res, or_jacobian_fn jac, const void* ctx, int64_t n,
                     double* U, double abs_tol, int max_newton, int restart, double gmres_rtol,
                     int* newton_iters, int* gmres_iters, double* final_norm) {
  double* R = (double*)malloc(sizeof(double) * n);
  double* d = (double*)malloc(sizeof(double) * n);
  int it = 0, gtot = 0, ok = 0;
  double rn = 0.0;
  for (;;) {
    res(ctx, U, R);
    rn = sqrt(dot(R, R, n));
    if (rn <= abs_tol) { ok = 1; break; }
    if (it >= max_newton) break;
    for (int64_t i = 0; i < n; ++i) { R[i] = -R[i]; d[i] = 0.0; }
    int gi = 0;
    const lin_ctx lc = {jac, ctx, U};
    gmres_op(apply_linearised, &lc, n, R, d, restart, 50 * restart, gmres_rtol, &gi);
    gtot += gi;
    for (int64_t i = 0; i < n; ++i) U[i] += d[i];
    ++it;
  }
  if (newton_iters) *newton_iters = it;
  if (gmres_iters) *gmres_iters = gtot;
  if (final_norm) *final_norm = rn;
  free(R);
  free(d);
  return ok;
}

typedef struct { const or_mesh* m; const or_params* p; double dt; const double* Un; } step_ctx;

static void res_implicit(const void* vctx, const double* U, double* R) {
  const step_ctx* c = (const step_ctx*)vctx;
  or_implicit_residual(c->m, c->p, c->dt, c->Un, U, R);
}

static void jac_implicit(const void* vctx, const double* U, const double* v, double* Jv) {
  const step_ctx* c = (const step_ctx*)vctx;
  or_implicit_jvp(c->m, c->p, c->dt, U, v, Jv);
}

/* Newton-Raphson on Eq. 14 (gradient-flow form). */
int or_newton(const or_mesh* m, const or_params* p, double dt, const double* Un, double* U,
              double abs_tol, int max_newton, int restart, double gmres_rtol,
              int* newton_iters, int* gmres_iters, double* final_norm) {
  const step_ctx ctx = {m, p, dt, Un};
  return newton_op(res_implicit, jac_implicit, &ctx, or_nnodes(m) * p->nf, U, abs_tol,
                   max_newton, restart, gmres_rtol, newton_iters, gmres_iters, final_norm);
}

/* ---- adjoint of the implicit Allen-Cahn trajectory (Supp. 2, Eq. II.1-II.6) --
 * Steps C(U^{n+1}; U^n, theta) = M (U^{n+1} - U^n)/dt + L r(U^{n+1}) = 0 from U^0,
 * objective O = (1/V) sum_i m_i U^N_i (the domain average, Eq. 19), parameters
 * theta = (L, kappa).  Reverse sweep with lambda^N = dO/dU^N:
 *   (dC/dU^{n+1})^T mu = lambda^{n+1}   (J = M/dt + L H symmetric: one GMRES solve)
 *   dO/dL     -= mu . r(U^{n+1})
 *   dO/dkappa -= mu . L K U^{n+1}
 *   lambda^n   = -(dC/dU^n)^T mu = M mu / dt
 * Newton steps to abs_tol; grads = [dO/dL, dO/dkappa].  Returns O. */
double or_implicit_adjoint(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                           const double* U0, double abs_tol, double* grads) {
  const int64_t NN = or_nnodes(m), n = NN * p->nf;
  double* traj = (double*)malloc(sizeof(double) * n * (nsteps + 1));
  double* mass = (double*)malloc(sizeof(double) * NN);
  double* lam = (double*)malloc(sizeof(double) * n);
  double* mu = (double*)malloc(sizeof(double) * n);
  double* t1 = (double*)malloc(sizeof(double) * n);
  or_lumped_mass(m, mass);
  double V = 0.0;
  for (int64_t i = 0; i < NN; ++i) V += mass[i];
  memcpy(traj, U0, sizeof(double) * n);
  for (int64_t s = 0; s < nsteps; ++s) {
    double* U = traj + (s + 1) * n;
    memcpy(U, traj + s * n, sizeof(double) * n);
    or_newton(m, p, dt, traj + s * n, U, abs_tol, 50, 30, 1e-12, NULL, NULL, NULL);
  }
  double O = 0.0;
  for (int f = 0; f < p->nf; ++f)
    for (int64_t i = 0; i < NN; ++i) {
      O += mass[i] * traj[nsteps * n + f * NN + i] / V;
      lam[f * NN + i] = mass[i] / V;
    }
  /* K U alone: the residual of the gradient energy with kappa = 1 and no local energy */
  or_params pK = *p;
  pK.kappa = 1.0;
  pK.W = 0.0;
  pK.alpha = pK.beta = pK.gamma = 0.0;
  grads[0] = grads[1] = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    const double* U = traj + (s + 1) * n;
    memset(mu, 0, sizeof(double) * n);
    or_gmres(m, p, dt, U, lam, mu, 30, 3000, 1e-13, NULL);
    or_residual(m, p, U, t1);  /* r(U) */
    grads[0] -= dot(mu, t1, n);
    or_residual(m, &pK, U, t1);  /* K U */
    grads[1] -= p->mob * dot(mu, t1, n);
    for (int f = 0; f < p->nf; ++f)
      for (int64_t i = 0; i < NN; ++i) lam[f * NN + i] = mass[i] * mu[f * NN + i] / dt;
  }
  free(traj); free(mass); free(lam); free(mu); free(t1);
  return O;
}

/* ---- implicit split Cahn-Hilliard (Eq. 9-10 with backward Euler, Eq. 13) --
 * Unknowns U = [c; mu] (2 N values), the previous composition cn:
 *   R_c  = M (c - cn) / dt + K_M mu
 *   R_mu = M mu - r(c)            (r = dE_h/dc: f'(c) by Gauss quadrature + kappa K c)
 * Jacobian action on v = [v_c; v_mu]:
 *   J_c  = M v_c / dt + K_M v_mu
 *   J_mu = M v_mu - H(c) v_c      (H the Hessian of E_h)  */
void or_chsplit_residual(const or_mesh* m, const or_params* p, double dt, const double* cn,
                         const double* U, double* R) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  or_mobility_stiffness_apply(m, p, U + NN, R);  /* K_M mu */
  or_residual(m, p, U, R + NN);                   /* r(c) */
  for (int64_t i = 0; i < NN; ++i) {
    R[i] += mass[i] * (U[i] - cn[i]) / dt;
    R[NN + i] = mass[i] * U[NN + i] - R[NN + i];
  }
  free(mass);
}

void or_chsplit_jvp(const or_mesh* m, const or_params* p, double dt, const double* U,
                    const double* v, double* Jv) {
  const int64_t NN = or_nnodes(m);
  double* mass = (double*)malloc(sizeof(double) * NN);
  or_lumped_mass(m, mass);
  or_mobility_stiffness_apply(m, p, v + NN, Jv);  /* K_M v_mu */
  or_hessian_apply(m, p, U, v, Jv + NN);           /* H(c) v_c */
  for (int64_t i = 0; i < NN; ++i) {
    Jv[i] += mass[i] * v[i] / dt;
    Jv[NN + i] = mass[i] * v[NN + i] - Jv[NN + i];
  }
  free(mass);
}

static void res_chsplit(const void* vctx, const double* U, double* R) {
  const step_ctx* c = (const step_ctx*)vctx;
  or_chsplit_residual(c->m, c->p, c->dt, c->Un, U, R);
}

static void jac_chsplit(const void* vctx, const double* U, const double* v, double* Jv) {
  const step_ctx* c = (const step_ctx*)vctx;
  or_chsplit_jvp(c->m, c->p, c->dt, U, v, Jv);
}

int or_chsplit_newton(const or_mesh* m, const or_params* p, double dt, const double* cn,
                      double* U, double abs_tol, int max_newton, int restart, double gmres_rtol,
                      int* newton_iters, int* gmres_iters, double* final_norm) {
  const step_ctx ctx = {m, p, dt, cn};
  return newton_op(res_chsplit, jac_chsplit, &ctx, 2 * or_nnodes(m), U, abs_tol, max_newton,
                   restart, gmres_rtol, newton_iters, gmres_iters, final_norm);
}

/* ---- discrete adjoint of the explicit Cahn-Hilliard map (Supp. 2) -------
 *
 * Forward map G(c; theta) = c - dt M_L^-1 K_M mu(c),  mu = M_L^-1 (F(c) + kappa K c),
 * with F(c)_i = sum_e sum_q w|J| f'(c_q) N_i and f = W c^2 (1-c)^2.
 * Loss = 1/2 sum_i m_i (c^N_i - c*_i)^2  (or 1/2 sum_i (c^N_i - c*_i)^2 when nodal_loss).
 * lambda^N = dLoss/dc^N; for n = N-1 .. 0 (lambda = lambda^{n+1}, c = c^n):
 *   y = M_L^-1 lambda,  z = K_M y,  w = M_L^-1 z
 *   dLoss/dM      += -dt z.mu / M            (K_M is linear in M)
 *   dLoss/dkappa  += -dt w.(K c)
 *   dLoss/dW      += -dt w.F(c) / W          (F is linear in W)
 *   dLoss/dm_a    += -dt M sum_e sum_q w|J| N_a(q) grad mu_q . grad y_q
 *   lambda^n = lambda - dt (F'(c) + kappa K) w        (F', K, K_M symmetric)
 * grad_scalars = [dkappa, dW, dM]; grad_mob_field (may be NULL); lambda0 = dLoss/dc^0
 * (may be NULL).  Returns the loss. */

typedef struct { const or_params* p; const double* mu; const double* y; double* g; } mobgrad_ctx;

static void mobgrad_elem(const or_mesh* m, const or_elem* e, const int64_t* nodes, void* vctx) {
  mobgrad_ctx* c = (mobgrad_ctx*)vctx;
  for (int q = 0; q < e->nq; ++q) {
    double mv, my, gm[3], gy[3];
    interp(e, nodes, c->mu, q, &mv, gm);
    interp(e, nodes, c->y, q, &my, gy);
    double dotg = 0.0;
    for (int k = 0; k < m->dim; ++k) dotg += gm[k] * gy[k];
    for (int a = 0; a < e->nn; ++a) c->g[nodes[a]] += e->wq * c->p->mob * e->N[q][a] * dotg;
  }
}

double or_ch_adjoint(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                     const double* c0, const double* target, int nodal_loss,
                     double* grad_scalars, double* grad_mob_field, double* lambda0) {
  const int64_t NN = or_nnodes(m);
  double* traj = (double*)malloc(sizeof(double) * NN * (nsteps + 1));
  double* mass = (double*)malloc(sizeof(double) * NN);
  double* mu = (double*)malloc(sizeof(double) * NN);
  double* lam = (double*)malloc(sizeof(double) * NN);
  double* y = (double*)malloc(sizeof(double) * NN);
  double* z = (double*)malloc(sizeof(double) * NN);
  double* w = (double*)malloc(sizeof(double) * NN);
  double* t1 = (double*)malloc(sizeof(double) * NN);
  double* gm = (double*)calloc(NN, sizeof(double));
  or_lumped_mass(m, mass);

  memcpy(traj, c0, sizeof(double) * NN);
  for (int64_t s = 0; s < nsteps; ++s) {
    memcpy(traj + (s + 1) * NN, traj + s * NN, sizeof(double) * NN);
    or_ch_explicit(m, p, dt, 1, traj + (s + 1) * NN);
  }
  const double* cN = traj + nsteps * NN;
  double loss = 0.0;
  for (int64_t i = 0; i < NN; ++i) {
    const double d = cN[i] - target[i];
    const double wgt = nodal_loss ? 1.0 : mass[i];
    loss += 0.5 * wgt * d * d;
    lam[i] = wgt * d;
  }

  or_params pK = *p;  /* K c alone: no local energy */
  pK.W = 0.0;
  pK.kappa = 1.0;
  or_params pF = *p;  /* F(c) alone: no gradient energy */
  pF.kappa = 0.0;
  double gk = 0.0, gW = 0.0, gM = 0.0;
  for (int64_t s = nsteps - 1; s >= 0; --s) {
    const double* c = traj + s * NN;
    or_ch_chemical_potential(m, p, c, mu);
    for (int64_t i = 0; i < NN; ++i) y[i] = lam[i] / mass[i];
    or_mobility_stiffness_apply(m, p, y, z);
    for (int64_t i = 0; i < NN; ++i) w[i] = z[i] / mass[i];
    gM += -dt * dot(z, mu, NN) / p->mob;
    or_residual(m, &pK, c, t1);
    gk += -dt * dot(w, t1, NN);
    or_residual(m, &pF, c, t1);
    gW += -dt * dot(w, t1, NN) / p->W;
    if (grad_mob_field) {
      mobgrad_ctx mc = {p, mu, y, gm};
      or_elem e;
      ref_element(m, &e);
      for_each_element(m, &e, mobgrad_elem, &mc);
    }
    or_hessian_apply(m, p, c, w, t1);
    for (int64_t i = 0; i < NN; ++i) lam[i] -= dt * t1[i];
  }
  if (grad_scalars) {
    grad_scalars[0] = gk;
    grad_scalars[1] = gW;
    grad_scalars[2] = gM;
  }
  if (grad_mob_field)
    for (int64_t i = 0; i < NN; ++i) grad_mob_field[i] = -dt * gm[i];
  if (lambda0) memcpy(lambda0, lam, sizeof(double) * NN);
  free(traj); free(mass); free(mu); free(lam); free(y); free(z); free(w); free(t1); free(gm);
  return loss;
}

/* ---- 3x3x3 convolution, stride 1, zero padding 1 (surrogate layers) -------
 * y[o][z][yy][x] = bias[o] + sum_{i, kz, ky, kx} w[o][i][kz][ky][kx] x[i][z+kz-1][yy+ky-1][x+kx-1]
 * with x = 0 outside the volume.  The two backward routines are the exact
 * transposes: dx = W^T dy and dW = dy x^T (summed over voxels), dbias = sum dy. */

static double xat(const double* x, int d, int h, int w, int i, int z, int y, int xx) {
  if (z < 0 || z >= d || y < 0 || y >= h || xx < 0 || xx >= w) return 0.0;
  return x[(((int64_t)i * d + z) * h + y) * w + xx];
}

void or_conv3d_fwd(const double* x, int ci, int d, int h, int w, const double* wt,
                   const double* bias, int co, double* y) {
#pragma omp parallel for collapse(2)
  for (int o = 0; o < co; ++o)
    for (int z = 0; z < d; ++z)
      for (int yy = 0; yy < h; ++yy)
        for (int xx = 0; xx < w; ++xx) {
          double s = bias ? bias[o] : 0.0;
          for (int i = 0; i < ci; ++i)
            for (int kz = 0; kz < 3; ++kz)
              for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx)
                  s += wt[((((int64_t)o * ci + i) * 3 + kz) * 3 + ky) * 3 + kx] *
                       xat(x, d, h, w, i, z + kz - 1, yy + ky - 1, xx + kx - 1);
          y[(((int64_t)o * d + z) * h + yy) * w + xx] = s;
        }
}

void or_conv3d_bwd_data(const double* dy, int co, int d, int h, int w, const double* wt, int ci,
                        double* dx) {
  /* dx[i][p] = sum_{o, k} w[o][i][k] dy[o][p - k + 1]  (the transpose of the forward map) */
#pragma omp parallel for collapse(2)
  for (int i = 0; i < ci; ++i)
    for (int z = 0; z < d; ++z)
      for (int yy = 0; yy < h; ++yy)
        for (int xx = 0; xx < w; ++xx) {
          double s = 0.0;
          for (int o = 0; o < co; ++o)
            for (int kz = 0; kz < 3; ++kz)
              for (int ky = 0; ky < 3; ++ky)
                for (int kx = 0; kx < 3; ++kx)
                  s += wt[((((int64_t)o * ci + i) * 3 + kz) * 3 + ky) * 3 + kx] *
                       xat(dy, d, h, w, o, z - kz + 1, yy - ky + 1, xx - kx + 1);
          dx[(((int64_t)i * d + z) * h + yy) * w + xx] = s;
        }
}

void or_conv3d_bwd_weight(const double* x, int ci, int d, int h, int w, const double* dy, int co,
                          double* dwt, double* dbias) {
#pragma omp parallel for collapse(2)
  for (int o = 0; o < co; ++o)
    for (int i = 0; i < ci; ++i)
      for (int k = 0; k < 27; ++k) {
        const int kz = k / 9, ky = (k / 3) % 3, kx = k % 3;
        double s = 0.0;
        for (int z = 0; z < d; ++z)
          for (int yy = 0; yy < h; ++yy)
            for (int xx = 0; xx < w; ++xx)
              s += dy[(((int64_t)o * d + z) * h + yy) * w + xx] *
                   xat(x, d, h, w, i, z + kz - 1, yy + ky - 1, xx + kx - 1);
        dwt[(((int64_t)o * ci + i) * 27) + k] = s;
      }
  if (dbias)
    for (int o = 0; o < co; ++o) {
      double s = 0.0;
      for (int64_t p = 0; p < (int64_t)d * h * w; ++p) s += dy[(int64_t)o * d * h * w + p];
      dbias[o] = s;
    }
}

/* threads of the OpenMP loops (<= 0: the runtime's default) */
void or_set_threads(int n) { omp_set_num_threads(n > 0 ? n : omp_get_num_procs()); }
