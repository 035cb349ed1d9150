/*
 * FP64 CPU oracle for the Q1 finite-element phase-field method (test
 * infrastructure only).
 *
 * Only the tests, the package's smoke check and the bench's CPU-baseline leg
 * use this library.  It shares no code, header, table or constant with the
 * CUDA path: the reference-element tables are built here from the
 * definitions (Q1 shape functions, 2-point Gauss rule per axis).
 *
 * Discretisation (JAX-PF, Sec. 2.2, Eq. 11-14):
 *   nodes on a uniform grid, n[0] x n[1] (x n[2]) nodes, spacing h[],
 *   Q1 elements, 2x2 (2x2x2) Gauss quadrature, zero-flux (natural) boundary
 *   conditions, lumped (row-sum) mass matrix.
 * Node numbering: node = (k*n[1] + j)*n[0] + i.  Multi-field arrays are
 * field-major: U[f*nnodes + node].
 *
 * Parity status per function is listed in the Python wrapper's docstring.
 */
#ifndef PF_ORACLE_H
#define PF_ORACLE_H
#include <stdint.h>

typedef struct {
  int dim;        /* 2 or 3 */
  int64_t n[3];   /* nodes per axis; n[2] = 1 in 2-D */
  double h[3];    /* node spacing per axis */
} or_mesh;

enum { OR_DOUBLE_WELL = 0, OR_FAN_CHEN = 1, OR_COUPLED = 2 };

typedef struct {
  int energy;               /* OR_DOUBLE_WELL or OR_FAN_CHEN */
  int nf;                   /* number of fields (order parameters) */
  double W;                 /* double-well height: f = W c^2 (1-c)^2 */
  double kappa;             /* gradient-energy coefficient */
  double mob;               /* scalar mobility (L for AC, M for CH) */
  double alpha, beta, gamma;/* Fan-Chen: f = sum(-a/2 e^2 + b/4 e^4) + g sum_{i<j} e_i^2 e_j^2 */
  const double* mob_field;  /* per-node mobility multiplier (CH), NULL = 1 */
  double mob2;              /* coupled AC-CH: M_eta (mob is M_c) */
} or_params;

int64_t or_nnodes(const or_mesh* m);
void or_lumped_mass(const or_mesh* m, double* mass);
double or_energy(const or_mesh* m, const or_params* p, const double* U);
void or_residual(const or_mesh* m, const or_params* p, const double* U, double* r);
void or_hessian_apply(const or_mesh* m, const or_params* p, const double* U,
                      const double* v, double* out);
void or_mobility_stiffness_apply(const or_mesh* m, const or_params* p,
                                 const double* mu, double* out);
void or_ac_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps, double* U);
void or_ch_chemical_potential(const or_mesh* m, const or_params* p, const double* c, double* mu);
void or_ch_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps, double* c);
/* Adjoint of an implicit Allen-Cahn trajectory: O = mean of U^N, grads = [dO/dL, dO/dkappa]. */
double or_implicit_adjoint(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                           const double* U0, double abs_tol, double* grads);
/* Implicit split Cahn-Hilliard: U = [c; mu] (2 planes), cn the previous c. */
void or_chsplit_residual(const or_mesh* m, const or_params* p, double dt, const double* cn,
                         const double* U, double* R);
void or_chsplit_jvp(const or_mesh* m, const or_params* p, double dt, const double* U,
                    const double* v, double* Jv);
int or_chsplit_newton(const or_mesh* m, const or_params* p, double dt, const double* cn,
                      double* U, double abs_tol, int max_newton, int restart, double gmres_rtol,
                      int* newton_iters, int* gmres_iters, double* final_norm);
/* Coupled Allen-Cahn / Cahn-Hilliard (Eq. 7, Supp. 3): U = [c; eta] (2 planes). */
void or_coupled_explicit(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                         double* U);
double or_mass_integral(const or_mesh* m, const double* c);
void or_implicit_residual(const or_mesh* m, const or_params* p, double dt, const double* Un,
                          const double* U, double* R);
void or_implicit_jvp(const or_mesh* m, const or_params* p, double dt, const double* U,
                     const double* v, double* Jv);
int or_gmres(const or_mesh* m, const or_params* p, double dt, const double* U, const double* b,
             double* x, int restart, int maxit, double rtol, int* iters_out);
int or_newton(const or_mesh* m, const or_params* p, double dt, const double* Un, double* U,
              double abs_tol, int max_newton, int restart, double gmres_rtol,
              int* newton_iters, int* gmres_iters, double* final_norm);
double or_ch_adjoint(const or_mesh* m, const or_params* p, double dt, int64_t nsteps,
                     const double* c0, const double* target, int nodal_loss,
                     double* grad_scalars, double* grad_mob_field, double* lambda0);
/* 3-D convolution with a 3x3x3 kernel, stride 1, zero padding of 1 (the layer
 * of the learned surrogate).  Layouts: x[c][d][h][w] (one sample), weights
 * w[co][ci][kz][ky][kx], bias[co]. */
void or_conv3d_fwd(const double* x, int ci, int d, int h, int w, const double* wt,
                   const double* bias, int co, double* y);
void or_conv3d_bwd_data(const double* dy, int co, int d, int h, int w, const double* wt, int ci,
                        double* dx);
void or_conv3d_bwd_weight(const double* x, int ci, int d, int h, int w, const double* dy, int co,
                          double* dwt, double* dbias);
/* ---- Eshelby inclusion: linear elasticity with a misfit eigenstrain
 * (Eq. 3-4, Supp. 3 Eq. III.1, objective Eq. 21-22); or_elastic.c.  dim 3,
 * displacements component-major u[c*nnodes + node]. ---- */
void or_elastic_lame(double E, double nu, double* lam, double* mu);
void or_elastic_apply(const or_mesh* m, double lam, double mu, const double* u, double* out);
void or_elastic_rhs(const or_mesh* m, double lam, double mu, double em, double el, double ea,
                    double* f);
double or_elastic_volume_functional(const or_mesh* m, double* g);
int or_elastic_cg(const or_mesh* m, double lam, double mu, const double* b, double* u,
                  double rtol, int maxit, int* iters);
double or_elastic_sensitivity(const or_mesh* m, double E, double nu, double em, double el,
                              double ea, const double* g, double rtol, int maxit, double* u_out,
                              double* grads);

/* threads of the OpenMP loops (<= 0: one per processor) */
void or_set_threads(int n);

#endif
