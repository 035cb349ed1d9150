"""CPU checks of the C ABI: the library builds, loads and exports every symbol
that include/pf.h declares; host-side argument validation needs no GPU."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "pf.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(pf_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def libpf():
    from paper_2601_06079_gb300 import build
    path = build.build()
    return C.CDLL(path)


def test_every_declared_symbol_is_exported(libpf):
    names = _declared()
    assert len(names) >= 7
    for n in names:
        assert hasattr(libpf, n), n


def test_binding_covers_header():
    from paper_2601_06079_gb300 import _lib
    assert sorted(_lib.exported_symbols()) == _declared()


def test_create_mesh_validates_on_host(libpf):
    from paper_2601_06079_gb300 import _lib
    _lib.lib()
    ok, ctx, ws = _lib.pf_create_mesh(2, [64, 64], [1.0, 1.0], _lib.PF_MODEL_CH, 1, 0)
    assert ok == 0 and ws >= 2 * 64 * 64 * 4
    # no workspace bound -> PF_ERR_STATE without touching the device
    assert _lib.pf_step_explicit(ctx, 0x1000, 1) == _lib.PF_ERR_STATE
    assert "workspace" in _lib.pf_last_error(ctx)
    assert _lib.pf_bind_workspace(ctx, 0x1001, ws) == _lib.PF_ERR_ARG  # misaligned
    st, ex = _lib.pf_explicit_workspace(ctx)
    assert st == 0 and 2 * 64 * 64 * 4 <= ex < ws
    assert _lib.pf_bind_workspace(ctx, 0x1000, ex - 1) == _lib.PF_ERR_ARG  # too small
    _lib.pf_destroy(ctx)
    for bad in ([1, 64], [64, 0]):
        st, _, _ = _lib.pf_create_mesh(2, bad, [1.0, 1.0], _lib.PF_MODEL_AC, 1, 0)
        assert st == _lib.PF_ERR_ARG
    st, _, _ = _lib.pf_create_mesh(2, [2, 8], [1.0, 1.0], _lib.PF_MODEL_CH, 1, 0)
    assert st == _lib.PF_ERR_ARG
    st, _, _ = _lib.pf_create_mesh(2, [8, 8], [1.0, -1.0], _lib.PF_MODEL_AC, 1, 0)
    assert st == _lib.PF_ERR_ARG
    _lib.pf_destroy(None)


def test_explicit_only_workspace_refuses_implicit_steps_on_host(libpf):
    # the explicit prefix serves explicit steps; the implicit step and the
    # implicit adjoint report PF_ERR_STATE before enqueueing anything
    from paper_2601_06079_gb300 import _lib
    _lib.lib()
    for dim, nodes, model in [(2, [64, 48], _lib.PF_MODEL_CH), (2, [64, 48], _lib.PF_MODEL_AC),
                              (3, [16, 16, 16], _lib.PF_MODEL_FANCHEN)]:
        st, ctx, ws = _lib.pf_create_mesh(dim, nodes, [1.0] * dim, model, 1, 0)
        assert st == 0
        st, ex = _lib.pf_explicit_workspace(ctx)
        assert st == 0 and 0 < ex < ws
        if dim == 3:  # one residual vector for the 3-D explicit step
            assert ex >= 16 ** 3 * 4
        assert _lib.pf_bind_workspace(ctx, 0x100000, ex) == 0
        assert _lib.pf_set_params(ctx, _lib.pf_params(1.0, 0.5, 1.0, 1e-3, 1.0, 1.0, 1.5,
                                                      0.5, None, 0.0)) == 0
        opts, stats = _lib.pf_newton_opts(20, 30, 300, 1e-5, 1e-3), _lib.pf_newton_stats()
        assert _lib.pf_step_implicit(ctx, 0x2000, 1, 0, opts, stats) == _lib.PF_ERR_STATE
        assert "explicit steps only" in _lib.pf_last_error(ctx)
        if model == _lib.PF_MODEL_CH:  # no implicit adjoint for the split CH system
            _lib.pf_destroy(ctx)
            continue
        nb = _lib.C.c_size_t(0)
        assert _lib.lib().pf_implicit_adjoint_workspace(ctx, 2, _lib.C.byref(nb)) == 0
        O, g = _lib.C.c_double(0), (_lib.C.c_double * 2)()
        st = _lib.lib().pf_implicit_adjoint(ctx, _lib.C.c_void_p(0x2000), 2, _lib.C.byref(opts),
                                            _lib.C.c_void_p(0x4000), nb.value, _lib.C.byref(O),
                                            g, _lib.C.byref(stats))
        assert st == _lib.PF_ERR_STATE
        _lib.pf_destroy(ctx)
    # an ensemble binds its whole workspace
    st, ctx, ws, _ = _lib.pf_create_ensemble([16, 8], [16, 12], None, 0)
    assert st == 0
    st, ex = _lib.pf_explicit_workspace(ctx)
    assert st == 0 and ex == ws
    _lib.pf_destroy(ctx)


def test_sq_distance_validates_on_host(libpf):
    # argument errors and the empty sum return before any CUDA call
    from paper_2601_06079_gb300 import _lib
    _lib.lib()
    assert _lib.pf_sq_distance(0, 0, 0, 0, 0) == (0, 0.0)
    assert _lib.pf_sq_distance(0x1000, 0x1000, -1, 0x2000, 0)[0] == _lib.PF_ERR_ARG
    for a, b, s in [(0, 0x1000, 0x2000), (0x1000, 0, 0x2000), (0x1000, 0x1000, 0)]:
        assert _lib.pf_sq_distance(a, b, 5, s, 0)[0] == _lib.PF_ERR_ARG
    v = _lib.C.c_double(1.0)
    assert _lib.lib().pf_sq_distance(None, None, 0, None, None, None) == _lib.PF_ERR_ARG
    assert _lib.lib().pf_sq_distance(None, None, 0, None, None, _lib.C.byref(v)) == 0
    assert v.value == 0.0


def test_sq_distance_wrapper_rejects_host_tensors(libpf):
    import torch

    import paper_2601_06079_gb300 as pf
    with pytest.raises(ValueError):
        pf.sq_distance(torch.zeros(4), torch.zeros(4))


def test_ensemble_calls_validate_on_host(libpf):
    # call order and parameter checks of the ensemble entry points return
    # before any CUDA call (a fake, never dereferenced workspace address)
    from paper_2601_06079_gb300 import _lib
    _lib.lib()
    st, ctx, ws, _ = _lib.pf_create_ensemble([16, 24], [16, 12], None, 0)
    assert st == 0
    good = _lib.pf_params(1.0, 0.5, 1.0, 1e-3, 0.0, 0.0, 0.0, 0.5, None, 0.0)
    # no workspace yet
    assert _lib.pf_set_ensemble_params(ctx, [good, good]) == _lib.PF_ERR_STATE
    assert _lib.pf_set_ensemble_schedule(ctx, [6, 6], None) == _lib.PF_ERR_STATE
    assert _lib.pf_tune_ensemble(ctx, 1, 2, 2)[0] == _lib.PF_ERR_STATE
    assert _lib.pf_bind_workspace(ctx, 0x100000, ws) == 0
    # parameters not set yet
    assert _lib.pf_set_ensemble_schedule(ctx, [6, 6], None) == _lib.PF_ERR_STATE
    assert _lib.pf_tune_ensemble(ctx, 1, 2, 2)[0] == _lib.PF_ERR_STATE
    bad_dt = _lib.pf_params(1.0, 0.5, 1.0, 0.0, 0.0, 0.0, 0.0, 0.5, None, 0.0)
    other_shift = _lib.pf_params(1.0, 0.5, 1.0, 1e-3, 0.0, 0.0, 0.0, 0.0, None, 0.0)
    with_field = _lib.pf_params(1.0, 0.5, 1.0, 1e-3, 0.0, 0.0, 0.0, 0.5, 0x2000, 0.0)
    for p in ([good, bad_dt], [good, other_shift], [with_field, good]):
        assert _lib.pf_set_ensemble_params(ctx, p) == _lib.PF_ERR_ARG
    _lib.pf_destroy(ctx)
    # a mesh context is not an ensemble
    st, ctx, ws = _lib.pf_create_mesh(2, [64, 64], [1.0, 1.0], _lib.PF_MODEL_AC, 1, 0)
    assert st == 0
    assert _lib.pf_set_ensemble_schedule(ctx, [6], None) == _lib.PF_ERR_ARG
    assert _lib.pf_tune_ensemble(ctx, 1, 1, 1)[0] == _lib.PF_ERR_ARG
    _lib.pf_destroy(ctx)
