"""GB300-native matrix-free phase-field solver (JAX-PF method, Q1 FEM).

Python face of libpf (include/pf.h).  PyTorch provides device memory and
streams only; every step of the method runs in the library's CUDA kernels.

    from paper_2601_06079_gb300 import Solver
    s = Solver((2048, 2048), h=1.0, model="ch")
    s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3, shift=0.5)
    s.step_explicit(c, 10_000)          # c: torch.float32 CUDA tensor (ny, nx)
    E, mass = s.energy(c)
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from ._lib import (PF_ENS_PER_STEP, PF_ENS_PERSISTENT, PF_ENS_PLAIN,  # noqa: F401
                   PF_MODEL_AC, PF_MODEL_CH, PF_MODEL_COUPLED, PF_MODEL_FANCHEN, pf_adjoint,
                   pf_adjoint_workspace, pf_barrier_selftest, pf_bind_workspace,
                   pf_explicit_workspace,
                   pf_create_ensemble, pf_create_mesh, pf_destroy, pf_set_ensemble_params,
                   pf_step_ensemble, pf_tune_ensemble, pf_set_ensemble_schedule,
                   pf_surrogate_param_count,
                   pf_surrogate_workspace, pf_surrogate_predict, pf_surrogate_train_step,
                   pf_conv3d_check, pf_surrogate_loss_grad,
                   pf_energy, pf_energy2d_static, pf_sq_distance, PF_SQ_DISTANCE_SCRATCH,
                   pf_implicit_residual, pf_jvp, pf_last_error, pf_set_params, pf_step_explicit,
                   pf_step_implicit)

_MODELS = {"ac": PF_MODEL_AC, "ch": PF_MODEL_CH, "fanchen": PF_MODEL_FANCHEN,
           "coupled": PF_MODEL_COUPLED}


def _on_stream(stream, nbytes, device, dtype=torch.uint8, shape=None):
    """Allocate a library buffer from the caching allocator's pool of `stream`,
    the stream that libpf enqueues its work on: the allocator then orders a
    later reuse of the block after that stream's work, not after torch's
    current stream's."""
    with torch.cuda.stream(stream):
        if shape is not None:
            return torch.empty(shape, dtype=dtype, device=device)
        return torch.empty(max(nbytes, 256), dtype=dtype, device=device)


class PFError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_lib.STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Solver:
    """One mesh + model + parameter set on one CUDA device and stream.

    shape: node counts (ny, nx) or (nz, ny, nx); h: spacing (scalar or per
    axis, x first); model: 'ac' | 'ch' | 'fanchen' | 'coupled' (2-D, state
    [c; eta] with n_fields = 2).  The workspace is a torch uint8 tensor owned
    by this object and bound to the library context: at first the part that
    explicit steps and diagnostics use (pf_explicit_workspace), grown to the
    whole workspace before the first implicit step or implicit adjoint.
    """

    def __init__(self, shape, h=1.0, model="ac", n_fields=1, device="cuda", stream=None):
        if model == "coupled":
            n_fields = 2
        self.shape = tuple(int(s) for s in shape)
        self.dim = len(self.shape)
        self.device = torch.device(device)
        if self.device.type != "cuda":
            raise ValueError("libpf runs on CUDA devices only")
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        hs = [float(h)] * self.dim if isinstance(h, (int, float)) else [float(v) for v in h]
        nodes = list(reversed(self.shape))
        self.n_fields = n_fields
        self.model = model
        st, self._ctx, ws = pf_create_mesh(self.dim, nodes, hs, _MODELS[model], n_fields,
                                           self.stream.cuda_stream)
        if st != 0:
            raise PFError(st, "pf_create_mesh rejected the mesh/model")
        self._ws_all = ws
        st, ws_explicit = pf_explicit_workspace(self._ctx)
        self._check(st)
        self._bind(ws_explicit)
        self._params = None
        self._keep = None

    def _bind(self, nbytes):
        self._ws = _on_stream(self.stream, nbytes, self.device)
        self._check(pf_bind_workspace(self._ctx, self._ws.data_ptr(), self._ws.numel()))

    def _implicit_workspace(self):
        """Grow the bound workspace to the implicit step's size (once)."""
        if self._ws.numel() < self._ws_all:
            self.stream.synchronize()  # earlier work may still use the old memory
            self._ws = None
            self._bind(self._ws_all)

    def _check(self, st):
        if st != 0:
            raise PFError(st, pf_last_error(self._ctx))

    def set_params(self, W=1.0, kappa=1.0, mobility=1.0, dt=0.01, shift=None,
                   alpha=1.0, beta=1.0, gamma=1.5, mobility_field=None, mobility2=0.0):
        """Material and step parameters.  Coupled model: mobility = M_c,
        mobility2 = M_eta, kappa = kappa_eta, shift applies to c."""
        if shift is None:
            shift = {"ac": 0.5, "ch": 0.5, "coupled": 0.6}.get(self.model, 0.0)
        mf = None
        if mobility_field is not None:
            mf = mobility_field.to(self.device, torch.float32).contiguous()
        p = _lib.pf_params(W, kappa, mobility, dt, alpha, beta, gamma, shift,
                           None if mf is None else mf.data_ptr(), mobility2)
        self._check(pf_set_params(self._ctx, p))
        self._params, self._keep = p, mf

    def _state(self, t):
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise ValueError("state must be a contiguous float32 CUDA tensor")
        want = self.n_fields * int(torch.tensor(self.shape).prod())
        if t.numel() != want:
            raise ValueError(f"state has {t.numel()} values, mesh needs {want}")
        return t.data_ptr()

    FORMS = {"fused_graph": _lib.PF_FORM_FUSED_GRAPH, "fused_stream": _lib.PF_FORM_FUSED_STREAM,
             "two_pass": _lib.PF_FORM_TWO_PASS}

    def set_form(self, form):
        """Execution form of the 2-D explicit step: 'fused_graph' (default),
        'fused_stream' (one launch per step) or 'two_pass' (the plain form)."""
        self._check(_lib.pf_set_form(self._ctx, self.FORMS[form]))

    def step_explicit(self, state, n_steps):
        """Advance `state` in place by n_steps explicit Euler steps (Eq. 12)."""
        self._check(pf_step_explicit(self._ctx, self._state(state), n_steps))
        return state

    def step_implicit(self, state, n_steps=1, guess=None, max_newton=20, gmres_restart=30,
                      gmres_max_iters=300, newton_rtol=1e-5, gmres_rtol=1e-3, check=True):
        """Backward-Euler steps (Eq. 13-14) by Newton-GMRES; returns the stats dict."""
        opts = _lib.pf_newton_opts(max_newton, gmres_restart, gmres_max_iters, newton_rtol,
                                   gmres_rtol)
        stats = _lib.pf_newton_stats()
        gp = self._state(guess) if guess is not None else 0
        self._implicit_workspace()
        st = pf_step_implicit(self._ctx, self._state(state), n_steps, gp, opts, stats)
        out = {k: getattr(stats, k) for k, _ in _lib.pf_newton_stats._fields_}
        if check:
            self._check(st)
        out["status"] = st
        return out

    def _vec(self, t):
        """A Newton-system vector: the state, or [c; mu] (two planes) for 2-D CH."""
        if self.model == "ch" and self.dim == 2:
            n = int(torch.tensor(self.shape).prod())
            if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()
                    and t.numel() == 2 * n):
                raise ValueError(f"2-D CH Newton vectors are [c; mu]: {2 * n} float32 values")
            return t.data_ptr()
        return self._state(t)

    def implicit_adjoint(self, U0, n_steps, max_newton=20, gmres_restart=30,
                         gmres_max_iters=300, newton_rtol=1e-5, gmres_rtol=1e-3):
        """Objective O = domain average of U^N after n_steps implicit steps from U0
        (Eq. 19) and its sensitivities {L, kappa} by the adjoint of Supp. 2
        (pf_implicit_adjoint).  Returns (O, grads, stats)."""
        C = _lib.C
        nb = C.c_size_t(0)
        self._check(_lib.lib().pf_implicit_adjoint_workspace(self._ctx, n_steps, C.byref(nb)))
        self._implicit_workspace()
        ws = _on_stream(self.stream, nb.value, self.device)
        opts = _lib.pf_newton_opts(max_newton, gmres_restart, gmres_max_iters, newton_rtol,
                                   gmres_rtol)
        O, g = C.c_double(0), (C.c_double * 2)()
        stats = _lib.pf_newton_stats()
        self._check(_lib.lib().pf_implicit_adjoint(self._ctx, C.c_void_p(self._state(U0)), n_steps,
                                                   C.byref(opts), C.c_void_p(ws.data_ptr()),
                                                   ws.numel(), C.byref(O), g, C.byref(stats)))
        return O.value, {"L": g[0], "kappa": g[1]}, {k: getattr(stats, k)
                                                     for k, _ in _lib.pf_newton_stats._fields_}

    def jvp(self, U, v, out=None):
        """J v of Eq. 14 (unscaled: includes the lumped mass); 2-D CH: the split
        system's Jacobian action on [v_c; v_mu] at [c; mu]."""
        out = torch.empty_like(v) if out is None else out
        self._check(pf_jvp(self._ctx, self._vec(U), self._vec(v), self._vec(out)))
        return out

    def implicit_residual(self, Un, U, out=None):
        """R = M (U - Un)/dt + L r(U) of Eq. 14; 2-D CH: the split system's
        residual at U = [c; mu] with Un = [c^n; (ignored)]."""
        out = torch.empty_like(U) if out is None else out
        self._check(pf_implicit_residual(self._ctx, self._vec(Un), self._vec(U),
                                         self._vec(out)))
        return out

    def adjoint(self, c0, target, n_steps, ckpt_every=100, nodal_loss=False, want_field=True,
                want_state=False):
        """Loss 1/2 sum w_i (c^N_i - target_i)^2 and its gradients by the discrete
        adjoint of the explicit CH map (2-D CH).  Returns (loss, grads) with grads
        = {kappa, W, M, mobility_field (float64 tensor), c0 (float32 tensor)}."""
        st, nbytes = pf_adjoint_workspace(self._ctx, n_steps, ckpt_every)
        self._check(st)
        ws = _on_stream(self.stream, nbytes, self.device)
        gm = (_on_stream(self.stream, 0, self.device, torch.float64, self.shape)
              if want_field else None)
        g0 = (_on_stream(self.stream, 0, self.device, torch.float32, self.shape)
              if want_state else None)
        st, loss, gs = pf_adjoint(self._ctx, self._state(c0), self._state(target), n_steps,
                                  ckpt_every, int(nodal_loss), ws.data_ptr(), ws.numel(),
                                  gm.data_ptr() if gm is not None else 0,
                                  g0.data_ptr() if g0 is not None else 0)
        self._check(st)
        return loss, {"kappa": gs[0], "W": gs[1], "M": gs[2], "mobility_field": gm, "c0": g0}

    def energy(self, state):
        """(E_h, mass integral) in FP64 (Eq. 5-6); synchronises the stream."""
        st, e, m = pf_energy(self._ctx, self._state(state))
        self._check(st)
        return e, m

    def close(self):
        if getattr(self, "_ctx", None):
            self.stream.synchronize()  # library work may still use the workspace
            pf_destroy(self._ctx)
            self._ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Ensemble:
    """A batch of independent 2-D Allen-Cahn meshes advanced together.

    shapes: list of (ny, nx); params: list of dicts (W, kappa, L, dt).  The
    packed state is one float32 CUDA tensor; instance i is
    state[offsets[i]:offsets[i+1]].view(shapes[i]).
    """

    MODES = {"persistent": PF_ENS_PERSISTENT, "per_step": PF_ENS_PER_STEP, "plain": PF_ENS_PLAIN}

    def __init__(self, shapes, device="cuda", stream=None):
        self.shapes = [tuple(int(v) for v in s) for s in shapes]
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        st, self._ctx, ws, self.offsets = pf_create_ensemble(
            [s[1] for s in self.shapes], [s[0] for s in self.shapes], None,
            self.stream.cuda_stream)
        if st != 0:
            raise PFError(st, "pf_create_ensemble rejected the instances")
        self._ws = _on_stream(self.stream, ws, self.device)
        self._check(pf_bind_workspace(self._ctx, self._ws.data_ptr(), self._ws.numel()))
        self.nclasses = len(set(self.shapes))

    def _check(self, st):
        if st != 0:
            raise PFError(st, pf_last_error(self._ctx))

    def set_params(self, params, shift=0.5):
        ps = [_lib.pf_params(p["W"], p["kappa"], p["L"], p["dt"], 1.0, 1.0, 1.5, shift, None)
              for p in params]
        self._check(pf_set_ensemble_params(self._ctx, ps))

    L2_POLICIES = ("normal", "stream", "stream_half")

    def candidates(self):
        """The tuner's schedule candidates in index order: (band rows, L2 policy)."""
        return [(ty, pol) for pol in self.L2_POLICIES for ty in (6, 12, 24)]

    def set_schedule(self, ty=None, l2=None):
        """Band height (6, 12, 24) and L2 policy ("normal", "stream",
        "stream_half") per instance (pf_set_ensemble_schedule); None keeps."""
        codes = None if l2 is None else [self.L2_POLICIES.index(p) for p in l2]
        self._check(pf_set_ensemble_schedule(self._ctx, ty, codes))

    def tune(self, reps=10):
        """Autotune (band height, L2 policy) per size class on the whole
        ensemble step (pf_tune_ensemble).  Returns (band height per instance,
        info) with info = {"l2": policy per instance, "uniform_us": {(ty,
        policy): us}, "tuned_us": .., "trials_us": per class (order of first
        appearance) {(ty, policy): us} of the candidates tried}."""
        st, ty, l2, us = pf_tune_ensemble(self._ctx, reps, len(self.shapes), self.nclasses)
        self._check(st)
        nc, cand = self.nclasses, self.candidates()
        trials = [{cand[j]: us[9 * c + j] for j in range(9) if us[9 * c + j] >= 0}
                  for c in range(nc)]
        return ty, {"l2": [self.L2_POLICIES[p] for p in l2],
                    "uniform_us": dict(zip(cand, us[9 * nc:9 * nc + 9])),
                    "tuned_us": us[9 * nc + 9], "trials_us": trials}

    def pack(self, fields):
        return torch.cat([torch.as_tensor(f, dtype=torch.float32).reshape(-1) for f in fields]
                         ).to(self.device).contiguous()

    def unpack(self, state):
        return [state[self.offsets[i]:self.offsets[i + 1]].view(self.shapes[i])
                for i in range(len(self.shapes))]

    def step(self, state, n_steps, mode="persistent"):
        if not (state.is_cuda and state.dtype == torch.float32 and state.is_contiguous()
                and state.numel() == self.offsets[-1]):
            raise ValueError("packed state must be a contiguous float32 CUDA tensor")
        self._check(pf_step_ensemble(self._ctx, state.data_ptr(), n_steps, self.MODES[mode]))
        return state

    def close(self):
        if getattr(self, "_ctx", None):
            self.stream.synchronize()  # library work may still use the workspace
            pf_destroy(self._ctx)
            self._ctx = None
            self._ws = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Surrogate:
    """Learned warm start for the implicit step (a 3-D conv U-Net, see
    pf_surrogate_* in include/pf.h).  Parameters live in FP32 CUDA tensors;
    init() draws them from a seeded He-normal recipe (output channels 8-15 and
    the input channels beyond 8 (history + 1) are zero and stay zero).

    history = 0: input U^n (8 channels), guess U^n + out_scale * net.
    history = 1: input [U^n; U^{n-1}], guess 2 U^n - U^{n-1} + s * net.
    history = 2: input [U^n; U^{n-1}; U^{n-2}], guess 3 U^n - 3 U^{n-1} + U^{n-2} + c * net.
    With history the inputs are the increments in units s = out_scale *
    RMS(U^n - U^{n-1}); the correction is in units of the last increment (s,
    linear extrapolation) or of the curvature (c = max(out_scale * RMS(U^n -
    2 U^{n-1} + U^{n-2}), 1e-3 s), quadratic extrapolation).  A
    history-2 network also accepts 16-channel inputs (its third-state weights
    then see zeros), which is how the second step of a run is predicted."""

    LAYERS = [(32, 32)] * 14 + [(32, 16)]

    def __init__(self, device="cuda", stream=None, history=0):
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self.history = int(history)
        st, self.n_params = pf_surrogate_param_count()
        if st != 0:
            raise PFError(st, "pf_surrogate_param_count")
        self.params = torch.zeros(self.n_params, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.step = 0
        self.out_scale = 1.0  # output unit (absolute without history, relative with it)
        self._ws = {}

    def init(self, seed=0, last_layer_scale=0.1):
        import numpy as np

        import pf_inputs as G
        chunks = []
        for l, (ci, co) in enumerate(self.LAYERS):
            used = 8 * (self.history + 1)
            fan_in = 27 * (used if l == 0 else ci)
            z = G.uniform(seed * 1000 + l, 27 * co * ci * 2, 0.0, 1.0, "surrogate")
            u1, u2 = np.maximum(z[0::2], 1e-12), z[1::2]
            normal = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)  # Box-Muller
            w = (normal * np.sqrt(2.0 / fan_in)).reshape(27, co, ci)
            if l == 0:
                w[:, :, used:] = 0.0
            if l == len(self.LAYERS) - 1:
                w *= last_layer_scale
                w[:, 8:, :] = 0.0
            chunks += [w.ravel(), np.zeros(co)]
        self.params.copy_(torch.from_numpy(np.concatenate(chunks).astype(np.float32)))
        self.m.zero_()
        self.v.zero_()
        self.step = 0

    def _workspace(self, batch, d, h, w, training):
        key = (batch, d, h, w, bool(training))
        if key not in self._ws:
            st, nb = pf_surrogate_workspace(batch, d, h, w, training)
            if st != 0:
                raise PFError(st, f"unsupported surrogate volume {key}")
            self._ws[key] = _on_stream(self.stream, nb, self.device)
        return self._ws[key]

    def _dims(self, x):
        b, nin, d, h, w = x.shape
        if nin % 8 or not 8 <= nin <= 8 * (self.history + 1):
            raise ValueError("input channels: 8 (U^n) times 1 + the states of history used")
        return b, nin, d, h, w

    def predict(self, x, out=None):
        """Guess for U^{n+1} ([batch][8][d][h][w]) from x ([batch][8 or 16][d][h][w],
        float32 CUDA); see the class docstring."""
        b, nin, d, h, w = self._dims(x)
        out = torch.empty((b, 8, d, h, w), device=x.device) if out is None else out
        ws = self._workspace(b, d, h, w, False)
        st = pf_surrogate_predict(self.params.data_ptr(), self.out_scale, x.data_ptr(), nin,
                                  out.data_ptr(), b, d, h, w, ws.data_ptr(), ws.numel(),
                                  self.stream.cuda_stream)
        if st != 0:
            raise PFError(st, "pf_surrogate_predict")
        return out

    def loss_grad(self, x, y, stiff=0.0):
        """(loss, gradient tensor) without an update; stiff weighs the error by
        (I + stiff K) (see pf_surrogate_train_step)."""
        b, nin, d, h, w = self._dims(x)
        ws = self._workspace(b, d, h, w, True)
        g = torch.empty_like(self.params)
        st, loss = pf_surrogate_loss_grad(self.params.data_ptr(), self.out_scale, x.data_ptr(),
                                          nin, y.data_ptr(), stiff, b, d, h, w, ws.data_ptr(),
                                          ws.numel(), self.stream.cuda_stream, g.data_ptr())
        if st != 0:
            raise PFError(st, "pf_surrogate_loss_grad")
        return loss, g

    def train_step(self, x, y, lr=1e-3, stiff=0.0):
        b, nin, d, h, w = self._dims(x)
        ws = self._workspace(b, d, h, w, True)
        self.step += 1
        st, loss = pf_surrogate_train_step(self.params.data_ptr(), self.out_scale,
                                           self.m.data_ptr(), self.v.data_ptr(), self.step, lr,
                                           x.data_ptr(), nin, y.data_ptr(), stiff, b, d, h, w,
                                           ws.data_ptr(), ws.numel(), self.stream.cuda_stream)
        if st != 0:
            raise PFError(st, "pf_surrogate_train_step")
        return loss


class Elastic:
    """Eshelby-inclusion elasticity (Eq. 3-4, eigenstrain of Supp. 3 Eq. III.1,
    objective Eq. 21-22; pf_elastic_* in include/pf.h) on a (nz, ny, nx) node
    grid.  Displacements are float32 CUDA tensors [3, nz, ny, nx]; the
    inclusion sits at node (0, 0, 0) with symmetry planes x, y, z = 0."""

    def __init__(self, shape, h=1.0, E=22.5, nu=0.3, m=0.01, l=0.5, a=20.0, device="cuda",
                 stream=None):
        assert len(shape) == 3
        self.shape = tuple(int(v) for v in shape)
        self.device = torch.device(device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        hs = (float(h),) * 3 if isinstance(h, (int, float)) else tuple(float(v) for v in h)
        self.e = _lib.pf_elastic((C.c_int64 * 3)(*reversed(self.shape)), (C.c_double * 3)(*hs),
                                 E, nu, m, l, a)
        self._ws = None
        self.stats = _lib.pf_cg_stats()

    def set(self, **kw):
        for k, v in kw.items():
            setattr(self.e, k, float(v))

    def _check(self, st, what):
        if st != 0:
            raise PFError(st, what)

    def _sp(self):
        return self.stream.cuda_stream

    def _workspace(self):
        if self._ws is None:
            st, n = _lib.pf_elastic_workspace(self.e)
            self._check(st, "pf_elastic_workspace")
            self._ws = _on_stream(self.stream, n, self.device)
        return self._ws

    def empty(self):
        return torch.empty((3,) + self.shape, dtype=torch.float32, device=self.device)

    def apply(self, u, out=None, constrain=False):
        out = self.empty() if out is None else out
        self._check(_lib.pf_elastic_apply(self.e, u.data_ptr(), out.data_ptr(), int(constrain),
                                          self._sp()), "pf_elastic_apply")
        return out

    def load(self, unit=False, out=None):
        out = self.empty() if out is None else out
        self._check(_lib.pf_elastic_load(self.e, int(unit), out.data_ptr(), self._sp()),
                    "pf_elastic_load")
        return out

    def solve(self, b=None, u=None, rtol=1e-6, max_iter=20000):
        u = self.empty() if u is None else u
        ws = self._workspace()
        self._check(_lib.pf_elastic_solve(self.e, b.data_ptr() if b is not None else None,
                                          u.data_ptr(), rtol, max_iter, ws.data_ptr(), ws.numel(),
                                          self._sp(), self.stats), "pf_elastic_solve")
        return u

    def sensitivity(self, g=None, u=None, rtol=1e-6, max_iter=20000):
        """(O, {"E": dO/dE, "nu": dO/dnu}, u), O = g . u or the volume V."""
        u = self.empty() if u is None else u
        ws = self._workspace()
        st, O, grads = _lib.pf_elastic_sensitivity(
            self.e, g.data_ptr() if g is not None else None, u.data_ptr(), rtol, max_iter,
            ws.data_ptr(), ws.numel(), self._sp(), self.stats)
        self._check(st, "pf_elastic_sensitivity")
        return O, {"E": grads[0], "nu": grads[1]}, u


class _CHMisfit(torch.autograd.Function):
    """Loss of an explicit CH trajectory with gradients from the library's
    hand-written adjoint kernels (forward computes loss and all gradients in
    one pf_adjoint call; backward scales them by the incoming gradient)."""

    @staticmethod
    def forward(ctx, mobility_field, kappa, W, M, c0, target, dt, n_steps, ckpt_every, h, nodal):
        shape = tuple(c0.shape)
        s = Solver(shape, h=h, model="ch", device=c0.device)
        s.set_params(W=float(W), kappa=float(kappa), mobility=float(M), dt=dt,
                     mobility_field=mobility_field.detach())
        loss, g = s.adjoint(c0.detach().contiguous(), target.detach().contiguous(), n_steps,
                            ckpt_every, nodal_loss=nodal, want_field=True, want_state=True)
        dev = c0.device
        ctx.save_for_backward(g["mobility_field"].to(mobility_field.dtype),
                              torch.tensor(g["kappa"], dtype=torch.float64, device=dev),
                              torch.tensor(g["W"], dtype=torch.float64, device=dev),
                              torch.tensor(g["M"], dtype=torch.float64, device=dev),
                              g["c0"])
        return torch.tensor(loss, dtype=torch.float64, device=dev)

    @staticmethod
    def backward(ctx, go):
        gm, gk, gw, gM, g0 = ctx.saved_tensors
        return (go * gm, (go * gk).to(torch.float64), (go * gw).to(torch.float64),
                (go * gM).to(torch.float64), (go * g0).to(g0.dtype), None, None, None, None,
                None, None)


def sq_distance(a, b, stream=None):
    """sum_i (a_i - b_i)^2 in FP64 for two contiguous float32 CUDA tensors of the
    same size (pf_sq_distance), enqueued on `stream` (torch's current stream by
    default)."""
    if a.dtype != torch.float32 or b.dtype != torch.float32 or not (a.is_cuda and b.is_cuda):
        raise ValueError("a and b must be float32 CUDA tensors")
    if a.numel() != b.numel() or not (a.is_contiguous() and b.is_contiguous()):
        raise ValueError("a and b must be contiguous and of the same size")
    stream = stream if stream is not None else torch.cuda.current_stream(a.device)
    scratch = _on_stream(stream, 0, a.device, dtype=torch.float64,
                         shape=(PF_SQ_DISTANCE_SCRATCH,))
    st, v = pf_sq_distance(a.data_ptr(), b.data_ptr(), a.numel(), scratch.data_ptr(),
                           stream.cuda_stream)
    if st != 0:
        raise PFError(st, "pf_sq_distance")
    return v


def ch_misfit(mobility_field, kappa, W, M, c0, target, dt, n_steps, ckpt_every=100, h=1.0,
              nodal_loss=False):
    """Differentiable CH trajectory misfit: 1/2 sum_i m_i (c^N_i - target_i)^2 after
    n_steps explicit steps from c0, as a function of the per-node mobility field
    and the scalars kappa, W, M (0-d tensors).  Gradients come from the discrete
    adjoint (pf_adjoint), not from autograd tracing."""
    return _CHMisfit.apply(mobility_field, kappa, W, M, c0, target, dt, n_steps, ckpt_every, h,
                           nodal_loss)
