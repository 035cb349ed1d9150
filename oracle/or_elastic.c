/*
 * FP64 oracle for the Eshelby-inclusion benchmark (test infrastructure only):
 * small-strain linear elasticity with a misfit eigenstrain, JAX-PF Eq. 3-4
 * (div sigma = 0, sigma = C : (eps - eps0)) with the eigenstrain of Supp. 3,
 * Eq. III.1, and the volume objective of Eq. 21 with its sensitivities to
 * Young's modulus and Poisson's ratio (Eq. 22).
 *
 * Discretisation: Q1 hexahedra on the uniform grid of or_mesh (dim 3), 2x2x2
 * Gauss quadrature, isotropic C with Lame constants lam, mu.  Displacements
 * are component-major: u[c*nn + node], c = 0, 1, 2 for x, y, z.
 *
 * Readings of the paper (it gives E and nu only):
 *  - eps0 = m phi(r) I with phi = (1 - tanh(l (r - a))) / 2, r = |x|: the
 *    inclusion factor is 1 inside (the paper prints 1/2 + 1/2 tanh, which is
 *    1 outside, while calling m the misfit inside the inclusion);
 *  - the inclusion sits at the corner x = 0 of the cube, so the planes x = 0,
 *    y = 0, z = 0 are symmetry planes (normal displacement zero) and the other
 *    faces are traction-free;
 *  - the volume is the small-strain one, V = int (1 + tr eps(u)) dOmega.
 * Everything here is plain element loops: the element stiffness is
 * integrated point by point from the shape-function gradients.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "pf_oracle.h"

#define NQ 8

static int64_t nn_of(const or_mesh* m) { return m->n[0] * m->n[1] * m->n[2]; }

static int64_t node_id(const or_mesh* m, int64_t i, int64_t j, int64_t k) {
  return (k * m->n[1] + j) * m->n[0] + i;
}

/* Gauss points on [0, 1] for one axis */
static double gpt(int q) { return q ? 0.5 + 0.5 / sqrt(3.0) : 0.5 - 0.5 / sqrt(3.0); }

/* gradients of the 8 trilinear shape functions of a box element with sides
   h at local point (s, t, w) in [0,1]^3; corner a = ax + 2 ay + 4 az */
static void shape_grad(double s, double t, double w, const double* h, double dN[8][3]) {
  for (int a = 0; a < 8; ++a) {
    const int ax = a & 1, ay = (a >> 1) & 1, az = a >> 2;
    const double Nx = ax ? s : 1.0 - s, Ny = ay ? t : 1.0 - t, Nz = az ? w : 1.0 - w;
    const double dx = (ax ? 1.0 : -1.0) / h[0], dy = (ay ? 1.0 : -1.0) / h[1],
                 dz = (az ? 1.0 : -1.0) / h[2];
    dN[a][0] = dx * Ny * Nz;
    dN[a][1] = Nx * dy * Nz;
    dN[a][2] = Nx * Ny * dz;
  }
}

/* element stiffness K_e[(a,i)][(b,j)], index a*3+i:
   int lam d_i N_a d_j N_b + mu (delta_ij grad N_a . grad N_b + d_j N_a d_i N_b) */
static void element_stiffness(const double* h, double lam, double mu, double Ke[24][24]) {
  memset(Ke, 0, sizeof(double) * 24 * 24);
  const double wq = h[0] * h[1] * h[2] / 8.0;
  for (int q = 0; q < NQ; ++q) {
    double dN[8][3];
    shape_grad(gpt(q & 1), gpt((q >> 1) & 1), gpt(q >> 2), h, dN);
    for (int a = 0; a < 8; ++a)
      for (int b = 0; b < 8; ++b) {
        const double gg = dN[a][0] * dN[b][0] + dN[a][1] * dN[b][1] + dN[a][2] * dN[b][2];
        for (int i = 0; i < 3; ++i)
          for (int j = 0; j < 3; ++j)
            Ke[a * 3 + i][b * 3 + j] +=
                wq * (lam * dN[a][i] * dN[b][j] + mu * ((i == j) * gg + dN[a][j] * dN[b][i]));
      }
  }
}

static int64_t elem_corner(const or_mesh* m, int64_t ex, int64_t ey, int64_t ez, int a) {
  return node_id(m, ex + (a & 1), ey + ((a >> 1) & 1), ez + (a >> 2));
}

/* out = K u (assembled over all elements of the mesh; no constraints).
   Elements are visited in 8 colours (parities of ex, ey, ez), so the threads of
   one colour never add into the same node. */
void or_elastic_apply(const or_mesh* m, double lam, double mu, const double* u, double* out) {
  const int64_t nn = nn_of(m);
  double Ke[24][24];
  element_stiffness(m->h, lam, mu, Ke);
  memset(out, 0, sizeof(double) * 3 * nn);
  const int64_t Ex = m->n[0] - 1, Ey = m->n[1] - 1, Ez = m->n[2] - 1;
  for (int colour = 0; colour < 8; ++colour) {
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t ez = cz; ez < Ez; ez += 2)
      for (int64_t ey = cy; ey < Ey; ey += 2)
        for (int64_t ex = cx; ex < Ex; ex += 2) {
          double ue[24], fe[24];
          for (int a = 0; a < 8; ++a) {
            const int64_t g = elem_corner(m, ex, ey, ez, a);
            for (int i = 0; i < 3; ++i) ue[a * 3 + i] = u[i * nn + g];
          }
          for (int r = 0; r < 24; ++r) {
            double s = 0.0;
            for (int c = 0; c < 24; ++c) s += Ke[r][c] * ue[c];
            fe[r] = s;
          }
          for (int a = 0; a < 8; ++a) {
            const int64_t g = elem_corner(m, ex, ey, ez, a);
            for (int i = 0; i < 3; ++i) out[i * nn + g] += fe[a * 3 + i];
          }
        }
  }
}

/* inclusion factor of Eq. III.1 (inclusion reading, see the header) */
static double incl(double r, double l, double a) { return 0.5 * (1.0 - tanh(l * (r - a))); }

/* f = int B^T C eps0: node a, component i gets
   sum_e sum_q w d_i N_a(q) (3 lam + 2 mu) m phi(x_q) */
void or_elastic_rhs(const or_mesh* m, double lam, double mu, double em, double el, double ea,
                    double* f) {
  const int64_t nn = nn_of(m);
  memset(f, 0, sizeof(double) * 3 * nn);
  const double wq = m->h[0] * m->h[1] * m->h[2] / 8.0;
  const double k3 = 3.0 * lam + 2.0 * mu;
  const int64_t Ex = m->n[0] - 1, Ey = m->n[1] - 1, Ez = m->n[2] - 1;
  for (int colour = 0; colour < 8; ++colour) {
    const int cx = colour & 1, cy = (colour >> 1) & 1, cz = colour >> 2;
#pragma omp parallel for collapse(2) schedule(static)
    for (int64_t ez = cz; ez < Ez; ez += 2)
      for (int64_t ey = cy; ey < Ey; ey += 2)
        for (int64_t ex = cx; ex < Ex; ex += 2)
          for (int q = 0; q < NQ; ++q) {
            const double s = gpt(q & 1), t = gpt((q >> 1) & 1), w = gpt(q >> 2);
            const double x = (ex + s) * m->h[0], y = (ey + t) * m->h[1], z = (ez + w) * m->h[2];
            const double sig0 = k3 * em * incl(sqrt(x * x + y * y + z * z), el, ea);
            double dN[8][3];
            shape_grad(s, t, w, m->h, dN);
            for (int a = 0; a < 8; ++a) {
              const int64_t g = elem_corner(m, ex, ey, ez, a);
              for (int i = 0; i < 3; ++i) f[i * nn + g] += wq * dN[a][i] * sig0;
            }
          }
  }
}

/* g with V = V0 + g . u, V0 the undeformed volume (returned):
   g_{a,i} = sum_e sum_q w d_i N_a(q), the quadrature of int tr eps(u) */
double or_elastic_volume_functional(const or_mesh* m, double* g) {
  const int64_t nn = nn_of(m);
  memset(g, 0, sizeof(double) * 3 * nn);
  const double wq = m->h[0] * m->h[1] * m->h[2] / 8.0;
  const int64_t Ex = m->n[0] - 1, Ey = m->n[1] - 1, Ez = m->n[2] - 1;
  for (int64_t ez = 0; ez < Ez; ++ez)
    for (int64_t ey = 0; ey < Ey; ++ey)
      for (int64_t ex = 0; ex < Ex; ++ex)
        for (int q = 0; q < NQ; ++q) {
          double dN[8][3];
          shape_grad(gpt(q & 1), gpt((q >> 1) & 1), gpt(q >> 2), m->h, dN);
          for (int a = 0; a < 8; ++a) {
            const int64_t gn = elem_corner(m, ex, ey, ez, a);
            for (int i = 0; i < 3; ++i) g[i * nn + gn] += wq * dN[a][i];
          }
        }
  return (double)Ex * m->h[0] * (double)Ey * m->h[1] * (double)Ez * m->h[2];
}

/* the symmetry-plane constraints: u_x = 0 on x = 0, u_y on y = 0, u_z on z = 0 */
static void zero_constrained(const or_mesh* m, double* v) {
  const int64_t nn = nn_of(m);
  for (int64_t k = 0; k < m->n[2]; ++k)
    for (int64_t j = 0; j < m->n[1]; ++j)
      for (int64_t i = 0; i < m->n[0]; ++i) {
        const int64_t g = node_id(m, i, j, k);
        if (i == 0) v[g] = 0.0;
        if (j == 0) v[nn + g] = 0.0;
        if (k == 0) v[2 * nn + g] = 0.0;
      }
}

void or_elastic_lame(double E, double nu, double* lam, double* mu) {
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *mu = E / (2.0 * (1.0 + nu));
}

static double dot(const double* a, const double* b, int64_t n) {
  double s = 0.0;
  for (int64_t i = 0; i < n; ++i) s += a[i] * b[i];
  return s;
}

/* Conjugate gradients for K u = b on the unconstrained degrees of freedom
   (constrained entries of b are ignored and of u set to zero), from u = 0,
   until |r| <= rtol |b|.  Returns 1 on convergence. */
int or_elastic_cg(const or_mesh* m, double lam, double mu, const double* b_in, double* u,
                  double rtol, int maxit, int* iters) {
  const int64_t n = 3 * nn_of(m);
  double* b = malloc(sizeof(double) * n);
  double* r = malloc(sizeof(double) * n);
  double* p = malloc(sizeof(double) * n);
  double* Ap = malloc(sizeof(double) * n);
  memcpy(b, b_in, sizeof(double) * n);
  zero_constrained(m, b);
  memset(u, 0, sizeof(double) * n);
  memcpy(r, b, sizeof(double) * n);
  memcpy(p, r, sizeof(double) * n);
  double rr = dot(r, r, n);
  const double stop = rtol * rtol * rr;
  int it = 0, ok = rr == 0.0;
  while (!ok && it < maxit) {
    or_elastic_apply(m, lam, mu, p, Ap);
    zero_constrained(m, Ap);
    const double alpha = rr / dot(p, Ap, n);
    for (int64_t i = 0; i < n; ++i) {
      u[i] += alpha * p[i];
      r[i] -= alpha * Ap[i];
    }
    const double rr1 = dot(r, r, n);
    ++it;
    if (rr1 <= stop) ok = 1;
    const double beta = rr1 / rr;
    for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];
    rr = rr1;
  }
  if (iters) *iters = it;
  free(b);
  free(r);
  free(p);
  free(Ap);
  return ok;
}

/* Objective O = g . u of the equilibrium displacement (K u = f(E, nu), f the
   eigenstrain load) and its sensitivities [dO/dE, dO/dnu] by the adjoint of the
   linear system (Supp. 2 with a stationary residual): K lambda = g, then
   dO/dtheta = lambda . (df/dtheta - dK/dtheta u), where dK/dtheta and
   df/dtheta are K and f with (lam, mu) replaced by their theta-derivatives.
   u_out (may be NULL) receives u.  Returns O; grads[2] gets the sensitivities. */
double or_elastic_sensitivity(const or_mesh* m, double E, double nu, double em, double el,
                              double ea, const double* g, double rtol, int maxit, double* u_out,
                              double* grads) {
  const int64_t n = 3 * nn_of(m);
  double lam, mu;
  or_elastic_lame(E, nu, &lam, &mu);
  double* f = malloc(sizeof(double) * n);
  double* u = malloc(sizeof(double) * n);
  double* la = malloc(sizeof(double) * n);
  double* t = malloc(sizeof(double) * n);
  double* ft = malloc(sizeof(double) * n);
  or_elastic_rhs(m, lam, mu, em, el, ea, f);
  or_elastic_cg(m, lam, mu, f, u, rtol, maxit, NULL);
  or_elastic_cg(m, lam, mu, g, la, rtol, maxit, NULL);
  const double O = dot(g, u, n);
  /* d(lam, mu)/dE and d(lam, mu)/dnu */
  const double D = (1.0 + nu) * (1.0 - 2.0 * nu);
  const double dl[2] = {nu / D, E * (1.0 + 2.0 * nu * nu) / (D * D)};
  const double dm[2] = {1.0 / (2.0 * (1.0 + nu)), -E / (2.0 * (1.0 + nu) * (1.0 + nu))};
  for (int k = 0; k < 2; ++k) {
    or_elastic_apply(m, dl[k], dm[k], u, t);
    or_elastic_rhs(m, dl[k], dm[k], em, el, ea, ft);
    for (int64_t i = 0; i < n; ++i) t[i] = ft[i] - t[i];
    zero_constrained(m, t);
    grads[k] = dot(la, t, n);
  }
  if (u_out) memcpy(u_out, u, sizeof(double) * n);
  free(f);
  free(u);
  free(la);
  free(t);
  free(ft);
  return O;
}
