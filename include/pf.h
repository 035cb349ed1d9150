/*
 * libpf -- GB300 (sm_103a) matrix-free phase-field solver, C ABI.
 *
 * Method (JAX-PF, Hu et al.): Q1 finite elements on a uniform grid, 2x2
 * (2x2x2) Gauss quadrature, lumped mass, zero-flux boundaries.  The
 * semi-discrete system is M dU/dt + r(U, theta) = 0 (Eq. 11) with
 *   r_i = sum_e sum_q w_q |J| [ f'(U_q) N_i(q) + kappa grad U_q . grad N_i(q) ]
 * (the gradient of the discrete free energy of Eq. 5-6).  Allen-Cahn
 * (Eq. 1) advances U <- U - dt L M^-1 r(U) (Eq. 12).  Cahn-Hilliard uses the
 * split form of Eq. 9-10, read as mu = f'(c) - kappa lap c:
 *   M mu = r(c),   c <- c - dt M^-1 K_M mu,
 * where K_M is the mobility-weighted stiffness matrix.  The implicit step
 * solves R(U) = M (U - U^n)/dt + L r(U) = 0 (Eq. 13-14) by Newton with a
 * matrix-free Jacobian-vector product inside GMRES.
 *
 * Conventions for every entry point:
 *   - Array arguments are DEVICE pointers to caller-owned memory unless the
 *     comment says "host".  Fields are FP32, structure-of-arrays: field f of
 *     a mesh with N nodes occupies state[f*N .. f*N+N-1]; node
 *     (i, j, k) sits at (k*ny + j)*nx + i (x fastest).
 *   - The library never allocates device memory.  pf_create_mesh reports the
 *     workspace size for every call (pf_explicit_workspace the smaller part
 *     that explicit steps need); the caller allocates it and binds it with
 *     pf_bind_workspace before any compute call.
 *   - Work is enqueued on the stream given at creation, in order, without a
 *     device synchronisation.  Calls that return host scalars (pf_energy,
 *     pf_step_implicit statistics, pf_adjoint) synchronise that stream.
 *   - Every call returns a pf_status; on failure pf_last_error(ctx) gives a
 *     message.  No C++ exception crosses the ABI.  After PF_ERR_CUDA the
 *     context should be destroyed.
 *   - A context is not thread-safe; use one per host thread.
 */
#ifndef PF_H
#define PF_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pf_ctx pf_ctx; /* opaque, owned by the library */

typedef enum {
  PF_OK = 0,
  PF_ERR_ARG = -1,            /* invalid argument (null pointer, size, model mismatch) */
  PF_ERR_CUDA = -2,           /* a CUDA runtime call or kernel launch failed */
  PF_ERR_NOT_CONVERGED = -3,  /* Newton / GMRES hit their iteration limits */
  PF_ERR_NONFINITE = -4,      /* a NaN or Inf was produced (e.g. dt above the stability bound) */
  PF_ERR_TIMEOUT = -5,        /* a bounded device-side wait expired */
  PF_ERR_STATE = -6           /* call order violated (no workspace bound, no params set) */
} pf_status;

typedef enum {
  PF_MODEL_AC = 0,      /* Allen-Cahn, double well f = W u^2 (1-u)^2 (Eq. 1, 5; Supp. 3) */
  PF_MODEL_CH = 1,      /* Cahn-Hilliard split form, same f (Eq. 2, 6, 9, 10) */
  PF_MODEL_FANCHEN = 2, /* n_fields Allen-Cahn order parameters, Fan-Chen grain-growth energy */
  PF_MODEL_COUPLED = 3  /* coupled Allen-Cahn / Cahn-Hilliard (Eq. 7 with the Supp. 3 polynomials
                           f_alpha, f_beta, h): fields [c; eta], 2-D explicit steps */
} pf_model;

typedef struct {
  double W;           /* double-well height (AC, CH) */
  double kappa;       /* gradient-energy coefficient (Eq. 5-6) */
  double mobility;    /* L (AC, Fan-Chen; Eq. 1 M_eta) or M (CH; Eq. 2 M_c) */
  double dt;          /* time step */
  double fc_alpha;    /* Fan-Chen f = sum_i(-a/2 e_i^2 + b/4 e_i^4) + g sum_{i<j} e_i^2 e_j^2 */
  double fc_beta;
  double fc_gamma;
  double shift;       /* the FP32 working state is stored as U - shift (exact change of
                         variable that keeps rounding relative to the deviation); 0.5 suits
                         the double well, 0 the Fan-Chen model */
  const float* mobility_field; /* 2-D CH only: device, one multiplier per node, M(x) = M m(x)
                                  interpolated by Q1 at Gauss points; NULL = uniform.
                                  Must stay valid while the context uses it.  With a field,
                                  pf_step_explicit uses the element form of K_M (tiled
                                  kernel) instead of the fused stencil kernel. */
  double mobility2;   /* COUPLED: M_eta, the order-parameter mobility (mobility is M_c,
                         kappa is kappa_eta, shift applies to c; W unused) */
} pf_params;

/* Newton-Krylov controls for the implicit step (Eq. 13-14).  NULL = defaults. */
typedef struct {
  int max_newton;       /* Newton corrections per time step (default 20) */
  int gmres_restart;    /* GMRES restart length m, 1..31 (default 30) */
  int gmres_max_iters;  /* GMRES iterations per Newton correction (default 300) */
  double newton_rtol;   /* stop when ||R||_2 <= newton_rtol * ||M U^n / dt||_2 (default 1e-5) */
  double gmres_rtol;    /* inexact-Newton forcing: GMRES stops at ||r|| <= max(gmres_rtol ||G||,
                           a tenth of the Newton target) (default 1e-3; no oversolving) */
} pf_newton_opts;

typedef struct {
  int newton_iters;         /* Newton corrections, summed over the call's steps */
  int gmres_iters;          /* GMRES iterations, summed */
  int converged;            /* 1 if every step met the Newton tolerance */
  double initial_residual;  /* ||R(U_0)||_2 of the first step's initial guess */
  double final_residual;    /* ||R||_2 at the end of the last step */
} pf_newton_stats;

/* Create a solver context for a uniform Q1 mesh.
 *   dim              2 (AC, CH: explicit and implicit steps, JVP, residual, energy
 *                    (CH implicit: the split system); COUPLED: explicit steps, n_fields = 2
 *                    planes [c; eta]) or 3 (AC with one field or FANCHEN: explicit and
 *                    implicit steps, JVP, residual)
 *   nodes[3]         nodes per axis (x, y, z); nodes[2] ignored in 2-D; each >= 2
 *                    (>= 3 along every axis for CH)
 *   h[3]             node spacing per axis (> 0)
 *   model, n_fields  n_fields must be 1 for AC/CH, 1..8 for FANCHEN
 *   stream           cudaStream_t (NULL = legacy default stream) on which all work runs
 *   workspace_bytes  out (host): device workspace that serves every call
 *                    (pf_explicit_workspace: the part explicit steps need)
 * Defines the discretisation of Sec. 2.2 / Eq. 11.  Host only; no CUDA call. */
pf_status pf_create_mesh(pf_ctx** out, int dim, const int64_t nodes[3], const double h[3],
                         pf_model model, int n_fields, void* stream, size_t* workspace_bytes);

/* Bytes of the leading part of the workspace that explicit steps (every form,
 * Eq. 12), pf_energy, pf_jvp, pf_implicit_residual and pf_adjoint use: the 2-D
 * working planes, the reduction buffers and, in 3-D, one residual vector.  The
 * implicit step's vectors (Eq. 14: iterate, U^n, correction, Krylov basis) take
 * the rest of workspace_bytes.  Host only; *bytes (host) out. */
pf_status pf_explicit_workspace(const pf_ctx* ctx, size_t* bytes);

/* Bind caller-owned device memory (256-byte aligned) as the context's scratch
 * space.  bytes >= the workspace_bytes of pf_create_mesh serves every call;
 * bytes >= pf_explicit_workspace serves every call but pf_step_implicit and
 * pf_implicit_adjoint, which then return PF_ERR_STATE (nothing enqueued) until a
 * full workspace is bound.  Smaller: PF_ERR_ARG.  Ensembles need their whole
 * workspace_bytes.  Binding again replaces the previous memory (captured CUDA
 * graphs are dropped).  The memory must outlive the context's use of it. */
pf_status pf_bind_workspace(pf_ctx* ctx, void* dev_ptr, size_t bytes);

/* Set the material and time-step parameters theta (Eq. 11, 15).  Host pointer p
 * is copied; p->mobility_field (device) is referenced, not copied. */
pf_status pf_set_params(pf_ctx* ctx, const pf_params* p);

/* Advance `state` (device, n_fields * N FP32, in/out) by n_steps >= 0 explicit
 * Euler steps with the lumped mass, Eq. 12: AC U <- U - dt L r(U)/m;
 * CH c <- c - dt K_M mu / m with m mu = r(c); COUPLED (Eq. 7) c <- c - dt M_c K mu / m
 * with m mu = dE/dc (no c gradient term) and eta <- eta - dt M_eta (dE/deta) / m, both
 * from the start of the step (one fused kernel per step, one launch per step).  2-D: one fused kernel per step
 * (see pf_set_form); 3-D: residual kernel then update.  Enqueues only. */
pf_status pf_step_explicit(pf_ctx* ctx, float* state, int64_t n_steps);

/* Execution form of the 2-D explicit step (AC and CH without a mobility field;
 * no counterpart in the paper, which has one array program).  All forms
 * compute the same discretisation in FP32 on the shifted state:
 *   PF_FORM_FUSED_GRAPH   one fused kernel per step, replayed from a CUDA graph
 *                         of 64 steps (default)
 *   PF_FORM_FUSED_STREAM  the same kernel, one launch per step from the host
 *   PF_FORM_TWO_PASS      the plain form: node-centric quadrature with index
 *                         reflection, CH's mu written to and read back from
 *                         HBM between two launches per step; the state buffer
 *                         doubles as the mu plane during the call.
 * PF_ERR_ARG for any other value.  Host only. */
enum { PF_FORM_FUSED_GRAPH = 0, PF_FORM_FUSED_STREAM = 1, PF_FORM_TWO_PASS = 2 };
pf_status pf_set_form(pf_ctx* ctx, int form);

/* Advance `state` (device, 3-D, 2-D Allen-Cahn or 2-D Cahn-Hilliard, in/out) by n_steps
 * backward-Euler steps, Eq. 13.  2-D Cahn-Hilliard solves the split system of
 * Eq. 9-10 for [c; mu]: R = [M (c - c^n)/dt + K_M mu;  M mu - r(c)] (state and
 * guess hold c alone; mu starts at M^-1 r of the starting c; the Newton target
 * is rtol ||M c^n / dt||; no per-node mobility field).  Otherwise:
 * each step solves R(U) = M (U - U^n)/dt + L r(U) = 0 (Eq. 14) by Newton, each
 * correction by restarted GMRES(m) on the Jacobian-vector product (matrix-free;
 * Krylov vectors FP32, inner products FP64, CGS2 orthogonalisation).
 * guess: device initial Newton iterate for the FIRST step (NULL = U^n); later
 * steps start from their U^n.  opts may be NULL (defaults); stats (host) may be
 * NULL.  Synchronises the stream.  PF_ERR_NOT_CONVERGED: state holds the last
 * iterate and stats the counts so far. */
pf_status pf_step_implicit(pf_ctx* ctx, float* state, int64_t n_steps, const float* guess,
                           const pf_newton_opts* opts, pf_newton_stats* stats);

/* Jacobian-vector product of Eq. 14 (3-D, or 2-D Allen-Cahn):
 * Jv = M v / dt + L (F''(U) v + kappa K v); 2-D Cahn-Hilliard: the split system's
 * J [v_c; v_mu] = [M v_c / dt + K_M v_mu;  M v_mu - H(c) v_c] on 2N-value vectors.
 * with F''(U) v = sum_e sum_q w|J| H_f(U_q) v_q N_i (the Hessian of the local
 * energy) and K the Q1 stiffness.  U, v, Jv: device, n_fields * N FP32.
 * Enqueues only. */
pf_status pf_jvp(pf_ctx* ctx, const float* U, const float* v, float* Jv);

/* Implicit residual of Eq. 14 (3-D, or 2-D Allen-Cahn): R = M (U - Un) / dt + L r(U);
 * 2-D Cahn-Hilliard: the split system's residual at U = [c; mu] (2N values) with the
 * first plane of Un = c^n.  Device arrays, n_fields * N FP32.  Enqueues only. */
pf_status pf_implicit_residual(pf_ctx* ctx, const float* Un, const float* U, float* R);

/* Bytes of caller-owned device workspace pf_implicit_adjoint needs for n_steps
 * steps: n_steps + 3 state vectors (every state of the trajectory is kept) and
 * 256 bytes.  Gradient-flow meshes only (3-D, 2-D Allen-Cahn).  Host only. */
pf_status pf_implicit_adjoint_workspace(pf_ctx* ctx, int64_t n_steps, size_t* bytes);

/* Sensitivities of an implicit trajectory by the adjoint method of Supp. 2
 * (Eq. II.1-II.6): n_steps backward-Euler steps (Eq. 13-14, Newton-GMRES with
 * opts, may be NULL) from U0 (device), objective O = (1/V) sum_i m_i U^N_i (the
 * domain average of Eq. 19), theta = (L, kappa).  Reverse sweep per step: one
 * GMRES solve of J(U^{n+1})^T mu = lambda^{n+1} (J = M/dt + L H is symmetric;
 * relative tolerance 1e-6, or opts->gmres_rtol where that is smaller),
 * dO/dL -= mu . r(U^{n+1}), dO/dkappa -= mu . L K U^{n+1}, lambda^n = M mu / dt.
 * objective, grads[2] = [dO/dL, dO/dkappa]: host.  workspace: device, >=
 * pf_implicit_adjoint_workspace bytes, 256-byte aligned.  stats (host, may be
 * NULL): forward Newton/GMRES counts plus the adjoint GMRES iterations.
 * Synchronises the stream. */
pf_status pf_implicit_adjoint(pf_ctx* ctx, const float* U0, int64_t n_steps,
                              const pf_newton_opts* opts, void* workspace, size_t bytes,
                              double* objective, double* grads, pf_newton_stats* stats);

/* Bytes of caller-owned device workspace pf_adjoint needs for n_steps steps
 * with a checkpoint every ckpt_every steps: (ceil(n_steps/ckpt_every) + 1)
 * checkpoint planes, ckpt_every segment planes, 3 more planes and small
 * reduction buffers.  2-D Cahn-Hilliard only. */
pf_status pf_adjoint_workspace(pf_ctx* ctx, int64_t n_steps, int ckpt_every, size_t* bytes);

/* Loss and gradients of the explicit 2-D Cahn-Hilliard trajectory (Eq. 12 with
 * the split form of Eq. 9-10 and the per-node mobility of pf_params), by the
 * discrete adjoint of the explicit map (sensitivities in the sense of Supp. 2,
 * Eq. II.1-II.6, taken through the time-stepping map):
 *   loss = 1/2 sum_i w_i (c_i^N - target_i)^2, w_i = m_i (nodal_loss = 0) or 1.
 * Forward: n_steps steps from state0 (device, not modified), storing the state
 * every ckpt_every steps; reverse: each segment is recomputed from its
 * checkpoint, then stepped backwards.
 *   adj_ws, adj_bytes   device workspace of pf_adjoint_workspace() bytes (256-aligned)
 *   loss                host, 1 double (may be NULL)
 *   grad_scalars        host, 3 doubles: dLoss/dkappa, dLoss/dW, dLoss/dM (may be NULL)
 *   grad_mobility       device, N doubles: dLoss/dm_i for the mobility field (may be NULL)
 *   grad_state0         device, N floats: dLoss/dc^0 (may be NULL)
 * With no mobility field bound the field is taken as 1 everywhere.  State and
 * adjoint are FP32, all gradient sums FP64.  Synchronises the stream. */
pf_status pf_adjoint(pf_ctx* ctx, const float* state0, const float* target, int64_t n_steps,
                     int ckpt_every, int nodal_loss, void* adj_ws, size_t adj_bytes, double* loss,
                     double* grad_scalars, double* grad_mobility, float* grad_state0);

/* Ensemble stepping modes for pf_step_ensemble. */
enum {
  PF_ENS_PERSISTENT = 0, /* one persistent launch for all steps (graph-captured), grid barrier */
  PF_ENS_PER_STEP = 1,   /* one launch per step covering every instance */
  PF_ENS_PLAIN = 2       /* the single-mesh fused step, one launch per instance and step */
};

/* Create a context for `count` independent 2-D Allen-Cahn instances (a batched
 * ensemble, the array-programming idea of Sec. 2.4 applied across whole
 * problems).  Instance i has nx[i] x ny[i] nodes (each >= 4) and spacing
 * h[2i], h[2i+1] (h may be NULL: 1).  States are packed: instance i occupies
 * offsets[i] .. offsets[i+1]-1 of one FP32 array (host out, count+1 entries).
 * Host only; reports the workspace size to bind with pf_bind_workspace. */
pf_status pf_create_ensemble(pf_ctx** out, int count, const int64_t* nx, const int64_t* ny,
                             const double* h, void* stream, size_t* workspace_bytes,
                             int64_t* offsets);

/* Per-instance parameters (host array of `count`; W, kappa, mobility = L, dt;
 * one shared shift; no mobility field).  Needs the workspace bound; copies the
 * per-instance arguments to the device and synchronises the stream. */
pf_status pf_set_ensemble_params(pf_ctx* ctx, const pf_params* params);

/* L2 policies of an ensemble instance's working planes: the eviction priority
 * its row loads and stores carry in the ensemble step.  Streaming a large
 * instance lets the lines of the others stay in L2 from step to step.  The
 * policy changes no result. */
enum {
  PF_L2_NORMAL = 0,      /* evict_normal */
  PF_L2_STREAM = 1,      /* evict_first */
  PF_L2_STREAM_HALF = 2  /* evict_first for half of the lines, the others unchanged */
};

/* Set the schedule of every instance: band height ty[i] (6, 12 or 24 rows per
 * warp task) and L2 policy l2[i] (PF_L2_*).  Either may be NULL (kept).  The
 * schedule changes no result.  Needs the workspace and parameters; uploads the
 * task list and synchronises the stream.  Out-of-range values: PF_ERR_ARG. */
pf_status pf_set_ensemble_schedule(pf_ctx* ctx, const int* ty, const int* l2);

/* Autotuner of the schedule per size class (no counterpart in the paper).
 * The candidates of a class are the 9 pairs (band height, L2 policy), index
 * j = 3 * policy + k with heights {6, 12, 24}[k].  Every candidate is timed
 * as the whole ensemble step (best of three back-to-back rounds of `reps`
 * per-step launches), the quantity the ensemble forms run.  First all classes
 * on one candidate, for each of the 9; then, from the best of those,
 * coordinate descent over the classes (most nodes first, at most three
 * passes), where a class takes another candidate only if the whole step gets
 * at least 1 % faster.  ty_out and l2_out (host, count) receive the choice per
 * instance; us_out (host, 9 * classes + 10 doubles, classes in order of first
 * appearance) the microseconds per step: [9 ci + j] with class ci on
 * candidate j during the descent (-1 where not tried), then the 9 uniform
 * candidates and the final choice.  Any of them may be NULL.  Overwrites the
 * working planes; synchronises the stream. */
pf_status pf_tune_ensemble(pf_ctx* ctx, int reps, int* ty_out, int* l2_out, double* us_out);

/* Advance every instance of the packed state (device, in/out) by n_steps
 * explicit steps (Eq. 12) in the given mode.  PF_ENS_PERSISTENT synchronises
 * the stream and returns PF_ERR_TIMEOUT if a grid-barrier wait expired
 * (about one second); the other modes only enqueue. */
pf_status pf_step_ensemble(pf_ctx* ctx, float* packed_state, int64_t n_steps, int mode);

/* Failure-detection self-test of the bounded grid barrier used by the persistent
 * ensemble: two co-resident blocks meet at a barrier that also expects
 * `phantom` (0 or 1) arrivals that never come.  phantom = 0 must return PF_OK;
 * phantom = 1 must return PF_ERR_TIMEOUT after about limit_cycles SM clocks,
 * with the context still usable.  dev_scratch: device, 3 unsigned ints. */
pf_status pf_barrier_selftest(unsigned* dev_scratch, long long limit_cycles, int phantom,
                              void* stream);

/* Discrete free energy E_h = sum_e sum_q w_q |J| [f(U_q) + kappa/2 |grad U_q|^2]
 * (Eq. 5-6) and, per field, the mass integral sum_i m_i U_i, accumulated in FP64.
 * energy: host, 1 double; mass: host, n_fields doubles (either may be NULL).
 * 2-D meshes.  Synchronises the stream. */
pf_status pf_energy(pf_ctx* ctx, const float* state, double* energy, double* mass);

/* Energy and mass of a 2-D single-field double-well state (AC or CH) without a
 * context or workspace, for callers that cannot allocate device memory: a
 * host that owns all device memory through its own allocator, a process held
 * to a fixed device-memory budget, or a latency-critical path where
 * cudaMalloc / cudaFree would synchronise the device.  The paper has no
 * counterpart; it computes the same E_h and sum_i m_i u_i as pf_energy.
 *   state         device, nx * ny FP32 values u (unshifted), node (i, j) at j*nx + i
 *   nx, ny        nodes per axis, >= 2, nx * ny <= 2^31 - 1 (else PF_ERR_ARG)
 *   hx, hy        node spacing (> 0);  W, kappa: f = W u^2 (1-u)^2, gradient coefficient
 *   out           device, 2 doubles: out[0] = E_h, out[1] = mass (written on `stream`)
 *   stream        cudaStream_t to enqueue on (NULL = legacy default stream)
 *   err           host, may be NULL: set to a static message ("" on success)
 * Allocates nothing: the reduction's scratch is a static device array of
 * 2 x 1024 doubles (16 KiB) inside libpf that every GPU loading the library
 * holds until exit.  The first call on each device looks up that array's
 * address on the current device; make it before any stream capture.  All
 * calls share the array and it keeps the last call's partial sums; nothing in
 * it needs to start at zero (each call overwrites every slot it reads), but
 * calls that overlap on the GPU (other streams, other threads) race on it and
 * must be serialised by the caller.  The looked-up address is cached per
 * device for the life of the process, so after cudaDeviceReset on a device
 * this entry point must not be called on that device again in the same
 * process (device memory it would write no longer exists).  Does not
 * synchronise; returns PF_ERR_CUDA if a launch fails. */
pf_status pf_energy2d_static(const float* state, int64_t nx, int64_t ny, double hx, double hy,
                             double W, double kappa, double* out, void* stream,
                             const char** err);

/* Squared distance sum_i (a_i - b_i)^2 of two FP32 device arrays: each
 * difference is formed in FP32 and its square split exactly into two FP32
 * terms; each thread sums them in a compensated FP32 pair (about 48 bits),
 * and the block and final sums run in FP64 in a fixed order, so repeated
 * calls give the same bits.  The learned warm start
 * takes sqrt(sum / n) over consecutive states U^{n+1} - U^n of its training
 * trajectories (Eq. 13 steps) as the output unit of a surrogate without
 * history.  No counterpart in the paper.
 *   a, b         device, n FP32 values each (may be NULL when n == 0)
 *   n            values, >= 0; n == 0 gives 0 and enqueues nothing
 *   dev_scratch  device, PF_SQ_DISTANCE_SCRATCH doubles owned by the caller;
 *                a call in flight on another stream must not share it
 *   stream       cudaStream_t to enqueue on (NULL = legacy default stream)
 *   out          host, 1 double
 * PF_ERR_ARG for a NULL out, n < 0 or (n > 0 and a NULL pointer); PF_ERR_CUDA
 * if a launch or the copy fails.  Synchronises the stream. */
enum { PF_SQ_DISTANCE_SCRATCH = 2050 };
pf_status pf_sq_distance(const float* a, const float* b, int64_t n, double* dev_scratch,
                         void* stream, double* out);

/* ---- Learned warm start for the implicit step (no counterpart in the paper) ----
 * A 3-D U-Net (4 levels, 32 channels, 3x3x3 convolutions, BF16 operands, FP32
 * accumulation; 15 layers) gives the first Newton iterate for U^{n+1}.
 * Parameters are an FP32 array of pf_surrogate_param_count() values: per layer
 * [27][c_out][c_in] weights then c_out biases, in layer order 32->32 x 14,
 * 32->16 (inputs padded to 32 channels, outputs 16 -> 8 used).
 * Inputs are planar FP32 [batch][n_in][d][h][w], the current state and up to
 * two earlier ones:
 *   n_in = 8:  x = U^n.  Guess = U^n + s * net, s = out_scale.
 *   n_in = 16: x = [U^n; U^{n-1}].  Guess = 2 U^n - U^{n-1} + s_b * net.
 *   n_in = 24: x = [U^n; U^{n-1}; U^{n-2}].  Guess = 3 U^n - 3 U^{n-1} + U^{n-2}
 *              + c_b * net.
 * With history the network sees U^n and the increments U^{n-k+1} - U^{n-k}
 * divided by s_b = out_scale * RMS_b(U^n - U^{n-1}) (per sample b, floored at
 * 1e-30): a learned correction to linear extrapolation in units of the last
 * increment, or to quadratic extrapolation in units of its curvature,
 * c_b = max(out_scale * RMS_b(U^n - 2 U^{n-1} + U^{n-2}), 1e-3 s_b), so that
 * the correction shrinks where the trajectory is nearly quadratic.  Outputs [batch][8][d][h][w]; d a multiple of 16, h and
 * w of 64.  out_scale must be positive and finite; anything else is PF_ERR_ARG. */
pf_status pf_surrogate_param_count(int64_t* n_params);

/* Device workspace bytes for one call on [batch][8][d][h][w] (training = 1 adds
 * the gradient buffers).  Host only. */
pf_status pf_surrogate_workspace(int batch, int d, int h, int w, int training, size_t* bytes);

/* out = the warm-start guess for U^{n+1} (see above).  All device pointers;
 * runs on `stream` and synchronises it.  Levels
 * whose (d, h) allow it (d even, h a multiple of 8) run the tcgen05 convolution;
 * PF_ERR_TIMEOUT if one of its bounded pipeline waits expired. */
pf_status pf_surrogate_predict(const float* params, float out_scale, const float* x, int n_in,
                               float* out, int batch, int d, int h, int w, void* workspace,
                               size_t bytes, void* stream);

/* One Adam step (lr, beta1 0.9, beta2 0.999, eps 1e-8; step >= 1 for the bias
 * correction) on the loss of the guess against y = U^{n+1} (planar
 * [batch][8][d][h][w]): with e the error field of the guess, in state units
 * for n_in = 8 and in units of s_b with history (every sample then weighs the
 * same whatever the size of its increment),
 *   loss = mean over nodes and fields of ((I + stiff K) e)^2,
 * K the assembled Q1 stiffness of the unit-spaced crop (natural boundary).
 * stiff = dt L kappa / h^2 weighs e the way the linear part of the implicit
 * Jacobian (Eq. 14) does, relative to its mass term; stiff = 0 is the plain
 * mean-squared error.  stiff < 0 or non-finite is PF_ERR_ARG.
 * params, adam_m, adam_v: device FP32 (updated in place); loss: host (may be
 * NULL; if given the stream is synchronised). */
pf_status pf_surrogate_train_step(float* params, float out_scale, float* adam_m, float* adam_v,
                                  int step, double lr, const float* x, int n_in, const float* y,
                                  double stiff, int batch, int d, int h, int w, void* workspace,
                                  size_t bytes, void* stream, double* loss);

/* Loss (as pf_surrogate_train_step) and its gradient with respect to every
 * parameter, written to grad (device FP32, pf_surrogate_param_count values),
 * without updating anything.  Workspace: pf_surrogate_workspace(..., training = 1).
 * loss: host (may be NULL; if given the stream is synchronised). */
pf_status pf_surrogate_loss_grad(const float* params, float out_scale, const float* x, int n_in,
                                 const float* y, double stiff, int batch, int d, int h, int w,
                                 void* workspace, size_t bytes, void* stream, double* loss,
                                 float* grad);

/* Single-layer probe of the surrogate's convolution kernels (tests): one sample,
 * planar FP32 [c][d][h][w]; weights [27][c_out][c_in] FP32 (rounded to BF16
 * inside).  (c_in, c_out) in {(16,32), (32,32), (32,16)}; d even, h and w
 * multiples of 8.  mode 0: out = conv(x) + bias; mode 1: out = conv^T(dy);
 * mode 2: out = [dW (27 x c_out x c_in), db (c_out)] for dy.  Modes 0, 1 and
 * 2 run the tcgen05 kernels (d even, h and w multiples of 8 -- always here);
 * modes 3, 4 and 6 are 0, 1 and 2 on the mma.sync kernels; mode 5 is the
 * failure-path self-test: mode 0 with no input copies issued, so every
 * bounded pipeline wait expires (about 2 s), the kernel frees its tensor
 * memory and returns, and the call reports PF_ERR_TIMEOUT with the context
 * still usable.  Workspace (256-byte aligned) of at least 2V(c_in + c_out) +
 * 4 * 27 c_in c_out + 128 V + 147,456 S bytes plus 256 per part (V = d h w,
 * S = the device's SM count: 22,413,312 bytes of partial sums on 152 SMs).
 * Synchronises the stream; PF_ERR_TIMEOUT if a tensor-core pipeline wait
 * expired. */
pf_status pf_conv3d_check(int mode, int cin, int cout, int d, int h, int w, const float* x,
                          const float* wt, const float* bias, const float* dy, float* out,
                          void* workspace, size_t bytes, void* stream);

/* ---- Eshelby inclusion: misfit elasticity (Eq. 3-4; eigenstrain Supp. 3
 * Eq. III.1; objective and sensitivities Eq. 21-22) ----
 * Small-strain isotropic elasticity on a uniform 3-D grid of Q1 hexahedra
 * (2x2x2 Gauss), div sigma = 0, sigma = C : (eps - eps0), with
 *   eps0 = m phi(r) I,  phi = (1 - tanh(l (r - a))) / 2,  r = |x|,
 * x measured from node (0, 0, 0).  The inclusion sits at that corner, so the
 * planes x = 0, y = 0, z = 0 are symmetry planes (normal displacement zero)
 * and the other faces are traction-free.  Displacements are FP32 device arrays
 * [3][nz][ny][nx] (x, y, z components, x fastest).  Context-free: every call
 * takes the problem description by pointer.  PF_ERR_ARG for n < 2, h <= 0,
 * E <= 0, nu outside (-1, 1/2) or non-finite m, l, a. */
typedef struct {
  int64_t n[3];  /* nodes per axis (x, y, z) */
  double h[3];   /* node spacing per axis */
  double E, nu;  /* Young's modulus, Poisson's ratio */
  double m, l, a;/* misfit strain, interface sharpness (1/length), inclusion radius */
} pf_elastic;

typedef struct {
  int iterations;      /* CG iterations (both solves for pf_elastic_sensitivity) */
  int converged;
  double initial_residual, final_residual; /* |r| of the (first) solve, FP64 */
} pf_cg_stats;

/* Device workspace bytes for pf_elastic_solve / pf_elastic_sensitivity (7
 * vectors of 3 nx ny nz floats plus scalars).  Host only. */
pf_status pf_elastic_workspace(const pf_elastic* e, size_t* bytes);

/* Ku = K u (matrix-free, all elements of the mesh); constrain = 1 zeroes the
 * rows of the symmetry-plane constraints.  u and Ku distinct device arrays.
 * Enqueued on `stream`, no synchronisation. */
pf_status pf_elastic_apply(const pf_elastic* e, const float* u, float* Ku, int constrain,
                           void* stream);

/* unit = 0: f = int B^T C eps0 (the eigenstrain load);  unit = 1: g with
 * V = V0 + g . u the small-strain volume int (1 + tr eps(u)) of Eq. 21.
 * No constraint applied.  Enqueued on `stream`. */
pf_status pf_elastic_load(const pf_elastic* e, int unit, float* f, void* stream);

/* Conjugate gradients for K u = b on the free degrees of freedom (b = NULL:
 * the eigenstrain load; b's constrained entries are ignored), from u = 0,
 * FP32 vectors and FP64 inner products, until |r| <= rtol |b| (checked every
 * 8 iterations) or max_iter.  Workspace 256-byte aligned, pf_elastic_workspace
 * bytes.  Synchronises the stream.  PF_ERR_NOT_CONVERGED at max_iter (u holds
 * the last iterate), PF_ERR_NONFINITE on a non-finite residual. */
pf_status pf_elastic_solve(const pf_elastic* e, const float* b, float* u, double rtol,
                           int max_iter, void* workspace, size_t bytes, void* stream,
                           pf_cg_stats* stats);

/* Objective O = g . u of the equilibrium displacement u (written to `u`) and
 * grads = [dO/dE, dO/dnu] by the adjoint of the linear system: K lambda = g,
 * dO/dtheta = lambda . (df/dtheta - dK/dtheta u).  g = NULL takes the volume
 * functional, and then O = V includes the undeformed volume V0.  With uniform
 * moduli u does not depend on E, and V does not depend on E or nu (the mean
 * strain of a traction-free body equals its mean eigenstrain), so those
 * sensitivities are zero up to the solver tolerance.  Same workspace, errors
 * and synchronisation as pf_elastic_solve; stats sum both solves. */
pf_status pf_elastic_sensitivity(const pf_elastic* e, const float* g, float* u, double rtol,
                                 int max_iter, void* workspace, size_t bytes, void* stream,
                                 double* objective, double* grads, pf_cg_stats* stats);

/* Human-readable description of the last failure on this context. */
/* Measured FP32 FMA throughput of the current device, in TFLOP/s (2 flop per
 * FMA).  No counterpart in the paper: it is the peak that the ALU-bound
 * kernels' rooflines are stated against (the bench measures it in the same
 * run).  Times a kernel of independent packed FP32 FMA chains on every SM
 * (best of three launches after a warm-up) on `stream` (cudaStream_t, NULL =
 * legacy default).  dev_sink: device, >= 4 bytes, that the kernel may write
 * (it keeps the chains from being optimised away).  tflops: host, 1 double.
 * PF_ERR_ARG for NULL pointers, PF_ERR_CUDA if a launch fails.  Synchronises
 * the stream. */
pf_status pf_fp32_peak(void* stream, float* dev_sink, double* tflops);

const char* pf_last_error(const pf_ctx* ctx);

/* Release the context (not the caller's workspace or arrays). NULL is a no-op. */
void pf_destroy(pf_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PF_H */
