"""Execution forms of the 2-D explicit step (fused + graph, fused per launch,
plain two-pass): each against the FP64 oracle at the same bar as the default
form, and against each other on the same inputs (ragged sizes, several tiles,
more than one graph replay)."""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu

FORMS = ["fused_graph", "fused_stream", "two_pass"]


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def run(model, u0, h, n_steps, form, **par):
    import paper_2601_06079_gb300 as pf
    s = pf.Solver(u0.shape, h=h, model=model)
    s.set_params(**par)
    s.set_form(form)
    t = torch.from_numpy(np.ascontiguousarray(u0, dtype=np.float32)).cuda()
    s.step_explicit(t, n_steps)
    torch.cuda.synchronize()
    return t.cpu().numpy()


@pytest.mark.parametrize("form", FORMS)
@pytest.mark.parametrize("shape", [(67, 131), (130, 61)])
def test_ch_forms_match_oracle(form, shape):
    c0 = G.ch_initial(3, shape)
    par = dict(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3)
    ref = O.Problem(shape, kappa=0.5, mob=1.0).ch_explicit(c0, 1e-3, 150)
    got = run("ch", c0, 1.0, 150, form, **par)
    assert rel_l2(got, ref) <= 1e-5


@pytest.mark.parametrize("form", FORMS)
def test_ac_forms_match_oracle_anisotropic(form):
    shape = (45, 77)
    u0 = G.ac_initial(4, shape)
    h = (0.9, 1.2)
    par = dict(W=1.3, kappa=0.7, mobility=1.1, dt=0.01)
    ref = O.Problem(shape, h=h, W=1.3, kappa=0.7, mob=1.1).ac_explicit(u0, 0.01, 130)
    got = run("ac", u0, h, 130, form, **par)
    assert rel_l2(got, ref) <= 1e-5


def test_forms_agree_with_each_other_on_2048():
    c0 = G.ch_initial(1, (2048, 2048))
    par = dict(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3)
    outs = [run("ch", c0, 1.0, 200, f, **par) for f in FORMS]
    for o in outs[1:]:
        assert rel_l2(o, outs[0]) <= 1e-6


def test_unknown_form_is_an_argument_error():
    import paper_2601_06079_gb300 as pf
    from paper_2601_06079_gb300 import _lib
    s = pf.Solver((16, 16), model="ch")
    assert _lib.pf_set_form(s._ctx, 3) == _lib.PF_ERR_ARG
