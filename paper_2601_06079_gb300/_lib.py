"""ctypes binding of libpf (include/pf.h): argument marshalling only.

Every function here keeps the C name and forwards to the shared library;
all arithmetic runs in the CUDA kernels behind it.  The library must be built
(``paper_2601_06079_gb300.build``); loading fails loudly otherwise -- there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

PF_OK = 0
PF_ERR_ARG = -1
PF_ERR_CUDA = -2
PF_ERR_NOT_CONVERGED = -3
PF_ERR_NONFINITE = -4
PF_ERR_TIMEOUT = -5
PF_ERR_STATE = -6

PF_MODEL_AC = 0
PF_MODEL_CH = 1
PF_MODEL_FANCHEN = 2
PF_MODEL_COUPLED = 3

PF_ENS_PERSISTENT = 0
PF_ENS_PER_STEP = 1
PF_ENS_PLAIN = 2

STATUS_NAMES = {0: "PF_OK", -1: "PF_ERR_ARG", -2: "PF_ERR_CUDA", -3: "PF_ERR_NOT_CONVERGED",
                -4: "PF_ERR_NONFINITE", -5: "PF_ERR_TIMEOUT", -6: "PF_ERR_STATE"}


class pf_params(C.Structure):
    _fields_ = [("W", C.c_double), ("kappa", C.c_double), ("mobility", C.c_double),
                ("dt", C.c_double), ("fc_alpha", C.c_double), ("fc_beta", C.c_double),
                ("fc_gamma", C.c_double), ("shift", C.c_double),
                ("mobility_field", C.c_void_p), ("mobility2", C.c_double)]


class pf_elastic(C.Structure):
    _fields_ = [("n", C.c_int64 * 3), ("h", C.c_double * 3), ("E", C.c_double),
                ("nu", C.c_double), ("m", C.c_double), ("l", C.c_double), ("a", C.c_double)]


class pf_cg_stats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int),
                ("initial_residual", C.c_double), ("final_residual", C.c_double)]


class pf_newton_opts(C.Structure):
    _fields_ = [("max_newton", C.c_int), ("gmres_restart", C.c_int), ("gmres_max_iters", C.c_int),
                ("newton_rtol", C.c_double), ("gmres_rtol", C.c_double)]


class pf_newton_stats(C.Structure):
    _fields_ = [("newton_iters", C.c_int), ("gmres_iters", C.c_int), ("converged", C.c_int),
                ("initial_residual", C.c_double), ("final_residual", C.c_double)]


_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libpf.so from the package's _build directory (never rebuilt here)."""
    global _LIB
    if _LIB is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(
                f"libpf is not built ({path} missing); run paper_2601_06079_gb300.build.build()")
        L = C.CDLL(path)
        ctx = C.c_void_p
        st = C.c_int
        L.pf_create_mesh.restype = st
        L.pf_create_mesh.argtypes = [C.POINTER(ctx), C.c_int, C.POINTER(C.c_int64),
                                     C.POINTER(C.c_double), C.c_int, C.c_int, C.c_void_p,
                                     C.POINTER(C.c_size_t)]
        L.pf_bind_workspace.restype = st
        L.pf_bind_workspace.argtypes = [ctx, C.c_void_p, C.c_size_t]
        L.pf_explicit_workspace.restype = st
        L.pf_explicit_workspace.argtypes = [ctx, C.POINTER(C.c_size_t)]
        L.pf_set_params.restype = st
        L.pf_set_params.argtypes = [ctx, C.POINTER(pf_params)]
        L.pf_step_explicit.restype = st
        L.pf_step_explicit.argtypes = [ctx, C.c_void_p, C.c_int64]
        L.pf_step_implicit.restype = st
        L.pf_step_implicit.argtypes = [ctx, C.c_void_p, C.c_int64, C.c_void_p,
                                       C.POINTER(pf_newton_opts), C.POINTER(pf_newton_stats)]
        L.pf_jvp.restype = st
        L.pf_jvp.argtypes = [ctx, C.c_void_p, C.c_void_p, C.c_void_p]
        L.pf_implicit_residual.restype = st
        L.pf_implicit_residual.argtypes = [ctx, C.c_void_p, C.c_void_p, C.c_void_p]
        L.pf_adjoint_workspace.restype = st
        L.pf_adjoint_workspace.argtypes = [ctx, C.c_int64, C.c_int, C.POINTER(C.c_size_t)]
        L.pf_adjoint.restype = st
        L.pf_adjoint.argtypes = [ctx, C.c_void_p, C.c_void_p, C.c_int64, C.c_int, C.c_int,
                                 C.c_void_p, C.c_size_t, C.POINTER(C.c_double),
                                 C.POINTER(C.c_double), C.c_void_p, C.c_void_p]
        L.pf_create_ensemble.restype = st
        L.pf_create_ensemble.argtypes = [C.POINTER(ctx), C.c_int, C.POINTER(C.c_int64),
                                         C.POINTER(C.c_int64), C.POINTER(C.c_double), C.c_void_p,
                                         C.POINTER(C.c_size_t), C.POINTER(C.c_int64)]
        L.pf_set_ensemble_params.restype = st
        L.pf_set_ensemble_params.argtypes = [ctx, C.POINTER(pf_params)]
        L.pf_set_ensemble_schedule.restype = st
        L.pf_set_ensemble_schedule.argtypes = [ctx, C.POINTER(C.c_int), C.POINTER(C.c_int)]
        L.pf_tune_ensemble.restype = st
        L.pf_tune_ensemble.argtypes = [ctx, C.c_int, C.POINTER(C.c_int), C.POINTER(C.c_int),
                                       C.POINTER(C.c_double)]
        L.pf_step_ensemble.restype = st
        L.pf_step_ensemble.argtypes = [ctx, C.c_void_p, C.c_int64, C.c_int]
        L.pf_barrier_selftest.restype = st
        L.pf_barrier_selftest.argtypes = [C.c_void_p, C.c_longlong, C.c_int, C.c_void_p]
        L.pf_surrogate_param_count.restype = st
        L.pf_surrogate_param_count.argtypes = [C.POINTER(C.c_int64)]
        L.pf_surrogate_workspace.restype = st
        L.pf_surrogate_workspace.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                             C.POINTER(C.c_size_t)]
        L.pf_surrogate_predict.restype = st
        L.pf_surrogate_predict.argtypes = [C.c_void_p, C.c_float, C.c_void_p, C.c_int, C.c_void_p,
                                           C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p,
                                           C.c_size_t, C.c_void_p]
        L.pf_surrogate_train_step.restype = st
        L.pf_surrogate_train_step.argtypes = [C.c_void_p, C.c_float, C.c_void_p, C.c_void_p,
                                              C.c_int, C.c_double, C.c_void_p, C.c_int,
                                              C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int,
                                              C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                              C.POINTER(C.c_double)]
        L.pf_surrogate_loss_grad.restype = st
        L.pf_surrogate_loss_grad.argtypes = [C.c_void_p, C.c_float, C.c_void_p, C.c_int,
                                             C.c_void_p, C.c_double, C.c_int, C.c_int, C.c_int,
                                             C.c_int, C.c_void_p, C.c_size_t, C.c_void_p,
                                             C.POINTER(C.c_double), C.c_void_p]
        L.pf_conv3d_check.restype = st
        L.pf_conv3d_check.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int,
                                      C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                      C.c_void_p, C.c_size_t, C.c_void_p]
        L.pf_energy.restype = st
        L.pf_energy.argtypes = [ctx, C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.pf_energy2d_static.restype = st
        L.pf_energy2d_static.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_double,
                                         C.c_double, C.c_double, C.c_double, C.c_void_p,
                                         C.c_void_p, C.POINTER(C.c_char_p)]
        L.pf_sq_distance.restype = st
        L.pf_sq_distance.argtypes = [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                     C.POINTER(C.c_double)]
        L.pf_implicit_adjoint_workspace.restype = st
        L.pf_implicit_adjoint_workspace.argtypes = [ctx, C.c_int64, C.POINTER(C.c_size_t)]
        L.pf_implicit_adjoint.restype = st
        L.pf_implicit_adjoint.argtypes = [ctx, C.c_void_p, C.c_int64, C.POINTER(pf_newton_opts),
                                          C.c_void_p, C.c_size_t, C.POINTER(C.c_double),
                                          C.POINTER(C.c_double), C.POINTER(pf_newton_stats)]
        L.pf_set_form.restype = st
        L.pf_set_form.argtypes = [ctx, C.c_int]
        L.pf_fp32_peak.restype = st
        L.pf_fp32_peak.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
        E = C.POINTER(pf_elastic)
        vp = C.c_void_p
        L.pf_elastic_workspace.restype = st
        L.pf_elastic_workspace.argtypes = [E, C.POINTER(C.c_size_t)]
        L.pf_elastic_apply.restype = st
        L.pf_elastic_apply.argtypes = [E, vp, vp, C.c_int, vp]
        L.pf_elastic_load.restype = st
        L.pf_elastic_load.argtypes = [E, C.c_int, vp, vp]
        L.pf_elastic_solve.restype = st
        L.pf_elastic_solve.argtypes = [E, vp, vp, C.c_double, C.c_int, vp, C.c_size_t, vp,
                                       C.POINTER(pf_cg_stats)]
        L.pf_elastic_sensitivity.restype = st
        L.pf_elastic_sensitivity.argtypes = [E, vp, vp, C.c_double, C.c_int, vp, C.c_size_t, vp,
                                             C.POINTER(C.c_double), C.POINTER(C.c_double),
                                             C.POINTER(pf_cg_stats)]
        L.pf_last_error.restype = C.c_char_p
        L.pf_last_error.argtypes = [ctx]
        L.pf_destroy.restype = None
        L.pf_destroy.argtypes = [ctx]
        _LIB = L
    return _LIB


def exported_symbols():
    """Names declared in include/pf.h (checked against the .so by the tests)."""
    return ["pf_create_mesh", "pf_explicit_workspace", "pf_bind_workspace", "pf_set_params",
            "pf_step_explicit",
            "pf_set_form",
            "pf_step_implicit", "pf_jvp", "pf_implicit_residual", "pf_adjoint_workspace",
            "pf_adjoint", "pf_implicit_adjoint_workspace", "pf_implicit_adjoint",
            "pf_create_ensemble", "pf_set_ensemble_params", "pf_set_ensemble_schedule",
            "pf_tune_ensemble",
            "pf_step_ensemble", "pf_barrier_selftest", "pf_surrogate_param_count",
            "pf_surrogate_workspace", "pf_surrogate_predict", "pf_surrogate_train_step",
            "pf_surrogate_loss_grad",
            "pf_conv3d_check", "pf_energy", "pf_elastic_workspace", "pf_elastic_apply",
            "pf_elastic_load", "pf_elastic_solve", "pf_elastic_sensitivity",
            "pf_energy2d_static", "pf_sq_distance", "pf_fp32_peak", "pf_last_error",
            "pf_destroy"]


# --- thin same-name wrappers -------------------------------------------------

def pf_create_mesh(dim, nodes, h, model, n_fields, stream):
    ctx = C.c_void_p()
    ws = C.c_size_t(0)
    n = (C.c_int64 * 3)(*(list(nodes) + [1] * (3 - len(nodes))))
    hh = (C.c_double * 3)(*(list(h) + [1.0] * (3 - len(h))))
    s = lib().pf_create_mesh(C.byref(ctx), dim, n, hh, model, n_fields, C.c_void_p(stream),
                             C.byref(ws))
    return s, ctx, ws.value


def pf_explicit_workspace(ctx):
    b = C.c_size_t(0)
    s = lib().pf_explicit_workspace(ctx, C.byref(b))
    return s, b.value


def pf_bind_workspace(ctx, ptr, nbytes):
    return lib().pf_bind_workspace(ctx, C.c_void_p(ptr), nbytes)


def pf_set_params(ctx, params: pf_params):
    return lib().pf_set_params(ctx, C.byref(params))


PF_FORM_FUSED_GRAPH, PF_FORM_FUSED_STREAM, PF_FORM_TWO_PASS = 0, 1, 2


def pf_set_form(ctx, form):
    return lib().pf_set_form(ctx, int(form))


def pf_fp32_peak(stream, sink_ptr):
    t = C.c_double(0.0)
    s = lib().pf_fp32_peak(C.c_void_p(stream), C.c_void_p(sink_ptr), C.byref(t))
    return s, t.value


def pf_step_explicit(ctx, state_ptr, n_steps):
    return lib().pf_step_explicit(ctx, C.c_void_p(state_ptr), int(n_steps))


def pf_step_implicit(ctx, state_ptr, n_steps, guess_ptr, opts, stats):
    return lib().pf_step_implicit(ctx, C.c_void_p(state_ptr), int(n_steps),
                                  C.c_void_p(guess_ptr) if guess_ptr else None,
                                  C.byref(opts) if opts is not None else None,
                                  C.byref(stats) if stats is not None else None)


def pf_jvp(ctx, U_ptr, v_ptr, out_ptr):
    return lib().pf_jvp(ctx, C.c_void_p(U_ptr), C.c_void_p(v_ptr), C.c_void_p(out_ptr))


def pf_implicit_residual(ctx, Un_ptr, U_ptr, out_ptr):
    return lib().pf_implicit_residual(ctx, C.c_void_p(Un_ptr), C.c_void_p(U_ptr),
                                      C.c_void_p(out_ptr))


def pf_adjoint_workspace(ctx, n_steps, ckpt_every):
    b = C.c_size_t(0)
    s = lib().pf_adjoint_workspace(ctx, int(n_steps), int(ckpt_every), C.byref(b))
    return s, b.value


def pf_adjoint(ctx, state0_ptr, target_ptr, n_steps, ckpt_every, nodal_loss, ws_ptr, ws_bytes,
               grad_mob_ptr, grad_state0_ptr):
    loss = C.c_double(0)
    gs = (C.c_double * 3)()
    s = lib().pf_adjoint(ctx, C.c_void_p(state0_ptr), C.c_void_p(target_ptr), int(n_steps),
                         int(ckpt_every), int(nodal_loss), C.c_void_p(ws_ptr), ws_bytes,
                         C.byref(loss), gs, C.c_void_p(grad_mob_ptr) if grad_mob_ptr else None,
                         C.c_void_p(grad_state0_ptr) if grad_state0_ptr else None)
    return s, loss.value, list(gs)


def pf_create_ensemble(nx, ny, h, stream):
    n = len(nx)
    ctx = C.c_void_p()
    ws = C.c_size_t(0)
    offs = (C.c_int64 * (n + 1))()
    hh = None if h is None else (C.c_double * (2 * n))(*[v for pair in h for v in pair])
    s = lib().pf_create_ensemble(C.byref(ctx), n, (C.c_int64 * n)(*nx), (C.c_int64 * n)(*ny), hh,
                                 C.c_void_p(stream), C.byref(ws), offs)
    return s, ctx, ws.value, list(offs)


def pf_set_ensemble_params(ctx, params):
    arr = (pf_params * len(params))(*params)
    return lib().pf_set_ensemble_params(ctx, arr)


def pf_set_ensemble_schedule(ctx, ty=None, l2=None):
    t = (C.c_int * len(ty))(*ty) if ty is not None else None
    p = (C.c_int * len(l2))(*l2) if l2 is not None else None
    return lib().pf_set_ensemble_schedule(ctx, t, p)


def pf_tune_ensemble(ctx, reps, count, nclasses):
    ty = (C.c_int * count)()
    l2 = (C.c_int * count)()
    us = (C.c_double * (9 * nclasses + 10))()
    s = lib().pf_tune_ensemble(ctx, reps, ty, l2, us)
    return s, list(ty), list(l2), list(us)


def pf_step_ensemble(ctx, state_ptr, n_steps, mode):
    return lib().pf_step_ensemble(ctx, C.c_void_p(state_ptr), int(n_steps), int(mode))


def pf_barrier_selftest(scratch_ptr, limit_cycles, phantom, stream):
    return lib().pf_barrier_selftest(C.c_void_p(scratch_ptr), int(limit_cycles), int(phantom),
                                     C.c_void_p(stream))


def pf_surrogate_param_count():
    n = C.c_int64(0)
    s = lib().pf_surrogate_param_count(C.byref(n))
    return s, n.value


def pf_surrogate_workspace(batch, d, h, w, training):
    b = C.c_size_t(0)
    s = lib().pf_surrogate_workspace(batch, d, h, w, int(training), C.byref(b))
    return s, b.value


def pf_surrogate_predict(params, out_scale, x, n_in, out, batch, d, h, w, ws, nbytes, stream):
    return lib().pf_surrogate_predict(C.c_void_p(params), out_scale, C.c_void_p(x), n_in,
                                      C.c_void_p(out), batch, d, h, w, C.c_void_p(ws), nbytes,
                                      C.c_void_p(stream))


def pf_surrogate_train_step(params, out_scale, m, v, step, lr, x, n_in, y, stiff, batch, d, h,
                            w, ws, nbytes, stream):
    loss = C.c_double(0)
    s = lib().pf_surrogate_train_step(C.c_void_p(params), out_scale, C.c_void_p(m), C.c_void_p(v),
                                      step, lr, C.c_void_p(x), n_in, C.c_void_p(y), stiff, batch,
                                      d, h, w, C.c_void_p(ws), nbytes, C.c_void_p(stream),
                                      C.byref(loss))
    return s, loss.value


def pf_surrogate_loss_grad(params, out_scale, x, n_in, y, stiff, batch, d, h, w, ws, nbytes,
                           stream, grad):
    loss = C.c_double(0)
    s = lib().pf_surrogate_loss_grad(C.c_void_p(params), out_scale, C.c_void_p(x), n_in,
                                     C.c_void_p(y), stiff, batch, d, h, w, C.c_void_p(ws), nbytes,
                                     C.c_void_p(stream), C.byref(loss), C.c_void_p(grad))
    return s, loss.value


def pf_conv3d_check(mode, cin, cout, d, h, w, x, wt, bias, dy, out, ws, nbytes, stream):
    return lib().pf_conv3d_check(mode, cin, cout, d, h, w, C.c_void_p(x), C.c_void_p(wt),
                                 C.c_void_p(bias) if bias else None,
                                 C.c_void_p(dy) if dy else None, C.c_void_p(out), C.c_void_p(ws),
                                 nbytes, C.c_void_p(stream))


def pf_energy(ctx, state_ptr):
    e, m = C.c_double(0), C.c_double(0)
    s = lib().pf_energy(ctx, C.c_void_p(state_ptr), C.byref(e), C.byref(m))
    return s, e.value, m.value


def pf_energy2d_static(state_ptr, nx, ny, hx, hy, W, kappa, out_ptr, stream):
    """Context-free energy/mass into a caller-owned device buffer of 2 doubles;
    returns (status, message)."""
    msg = C.c_char_p()
    s = lib().pf_energy2d_static(C.c_void_p(state_ptr), nx, ny, hx, hy, W, kappa,
                                 C.c_void_p(out_ptr), C.c_void_p(stream), C.byref(msg))
    return s, (msg.value.decode() if msg.value else "")


PF_SQ_DISTANCE_SCRATCH = 2050


def pf_sq_distance(a_ptr, b_ptr, n, scratch_ptr, stream):
    """sum_i (a_i - b_i)^2 of two device FP32 arrays; returns (status, value)."""
    v = C.c_double(0.0)
    s = lib().pf_sq_distance(C.c_void_p(a_ptr), C.c_void_p(b_ptr), n, C.c_void_p(scratch_ptr),
                             C.c_void_p(stream), C.byref(v))
    return s, v.value


def pf_elastic_workspace(e):
    n = C.c_size_t(0)
    s = lib().pf_elastic_workspace(C.byref(e), C.byref(n))
    return s, n.value


def pf_elastic_apply(e, u, Ku, constrain, stream):
    return lib().pf_elastic_apply(C.byref(e), C.c_void_p(u), C.c_void_p(Ku), int(constrain),
                                  C.c_void_p(stream))


def pf_elastic_load(e, unit, f, stream):
    return lib().pf_elastic_load(C.byref(e), int(unit), C.c_void_p(f), C.c_void_p(stream))


def pf_elastic_solve(e, b, u, rtol, max_iter, ws, nbytes, stream, stats):
    return lib().pf_elastic_solve(C.byref(e), C.c_void_p(b) if b else None, C.c_void_p(u),
                                  float(rtol), int(max_iter), C.c_void_p(ws), nbytes,
                                  C.c_void_p(stream), C.byref(stats))


def pf_elastic_sensitivity(e, g, u, rtol, max_iter, ws, nbytes, stream, stats):
    obj = C.c_double(0.0)
    grads = (C.c_double * 2)()
    s = lib().pf_elastic_sensitivity(C.byref(e), C.c_void_p(g) if g else None, C.c_void_p(u),
                                     float(rtol), int(max_iter), C.c_void_p(ws), nbytes,
                                     C.c_void_p(stream), C.byref(obj), grads, C.byref(stats))
    return s, obj.value, [grads[0], grads[1]]


def pf_last_error(ctx) -> str:
    r = lib().pf_last_error(ctx)
    return r.decode() if r else ""


def pf_destroy(ctx):
    lib().pf_destroy(ctx)
