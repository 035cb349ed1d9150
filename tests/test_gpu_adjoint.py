"""GPU parity of the CH forward step with a per-node mobility field and of the
discrete adjoint (gradients w.r.t. kappa, W, M and the mobility field) against
the FP64 oracle, whose adjoint is pinned to central finite differences by the
CPU tests.  Gradient bar: relative error <= 1e-4."""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu
GRAD = 1e-4


def _pf():
    import paper_2601_06079_gb300 as pf
    return pf


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def setup(shape, width=(2.0, 5.0), kappa=0.6, W=1.1, M=0.9, seed=3):
    mob = G.gaussian_mobility(seed, shape, h=1.0, width=width)
    c0 = G.ch_initial(seed + 1, shape)
    target = G.ch_initial(seed + 2, shape)
    pf = _pf()
    s = pf.Solver(shape, model="ch")
    s.set_params(W=W, kappa=kappa, mobility=M, dt=0.02, mobility_field=cu(mob))
    P = O.Problem(shape, W=W, kappa=kappa, mob=M, mob_field=mob)
    return s, P, mob, c0, target


@pytest.mark.parametrize("shape,steps", [((3, 4), 20), ((37, 45), 50), ((130, 67), 100)])
def test_forward_with_mobility_field_matches_oracle(shape, steps):
    s, P, mob, c0, _ = setup(shape)
    t = cu(c0)
    s.step_explicit(t, steps)
    ref = P.ch_explicit(c0, 0.02, steps)
    assert rel(t.cpu().numpy(), ref) <= 1e-5


@pytest.mark.parametrize("shape,steps,ck", [((24, 20), 30, 7), ((48, 40), 60, 25)])
def test_adjoint_matches_oracle_adjoint(shape, steps, ck):
    s, P, mob, c0, target = setup(shape)
    loss, g = s.adjoint(cu(c0), cu(target), steps, ck, want_state=True)
    oloss, og = P.ch_adjoint(c0, target, 0.02, steps)
    assert abs(loss - oloss) <= 1e-5 * abs(oloss)
    for k in ("kappa", "W", "M"):
        assert abs(g[k] - og[k]) <= GRAD * abs(og[k]), (k, g[k], og[k])
    assert rel(g["mobility_field"].cpu().numpy(), og["mob_field"]) <= GRAD
    assert rel(g["c0"].cpu().numpy(), og["c0"]) <= GRAD


def test_adjoint_nodal_loss_and_uniform_mobility():
    shape = (21, 26)
    pf = _pf()
    c0, target = G.ch_initial(5, shape), G.ch_initial(6, shape)
    s = pf.Solver(shape, model="ch")
    s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=0.02)
    loss, g = s.adjoint(cu(c0), cu(target), 40, 9, nodal_loss=True)
    P = O.Problem(shape, W=1.0, kappa=0.5, mob=1.0, mob_field=np.ones(shape))
    oloss, og = P.ch_adjoint(c0, target, 0.02, 40, nodal_loss=True)
    assert abs(loss - oloss) <= 1e-5 * abs(oloss)
    for k in ("kappa", "W", "M"):
        assert abs(g[k] - og[k]) <= GRAD * abs(og[k]), k
    assert rel(g["mobility_field"].cpu().numpy(), og["mob_field"]) <= GRAD


def test_checkpoint_interval_does_not_change_the_result():
    s, _, _, c0, target = setup((33, 29))
    outs = [s.adjoint(cu(c0), cu(target), 45, ck) for ck in (1, 7, 45, 100)]
    for loss, g in outs[1:]:
        assert loss == outs[0][0]
        assert g["kappa"] == outs[0][1]["kappa"] and g["M"] == outs[0][1]["M"]
        assert torch.equal(g["mobility_field"], outs[0][1]["mobility_field"])


@pytest.mark.parametrize("n,steps", [(128, 400), (512, 2000)])
def test_calibration_config_against_oracle_adjoint(n, steps):
    # 2-D CH with an 8-Gaussian mobility field; the target comes from the
    # oracle run with the hidden (kappa, M, W) = (0.6, 0.8, 1.1) and its own
    # hidden field.  n = 512 with 2,000 steps and a checkpoint every 100 is the
    # calibration workload; the oracle's discrete adjoint (pinned to central
    # differences on the CPU) holds the whole FP64 trajectory, about 4.2 GB.
    shape = (n, n)
    mob = G.gaussian_mobility(1, shape, h=1.0)
    mob_hidden = G.gaussian_mobility(2, shape, h=1.0)
    c0 = G.ch_initial(1, shape)
    O.set_threads(0)
    target = O.Problem(shape, W=1.1, kappa=0.6, mob=0.8, mob_field=mob_hidden).ch_explicit(
        c0, 1e-3, steps)
    target32 = target.astype(np.float32)
    pf = _pf()
    s = pf.Solver(shape, model="ch")
    s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3, mobility_field=cu(mob))
    loss, g = s.adjoint(cu(c0), cu(target32), steps, 100)
    P = O.Problem(shape, W=1.0, kappa=0.5, mob=1.0, mob_field=mob)
    oloss, og = P.ch_adjoint(c0, target32, 1e-3, steps)
    assert oloss > 0
    errs = {k: abs(g[k] - og[k]) / abs(og[k]) for k in ("kappa", "W", "M")}
    errs["mobility_field"] = rel(g["mobility_field"].cpu().numpy(), og["mob_field"])
    print(f"calibration {n}^2 x {steps}: loss rel {abs(loss - oloss) / oloss:.2e}, grads", errs)
    assert abs(loss - oloss) <= 1e-4 * abs(oloss)
    for k, e in errs.items():
        assert e <= GRAD, (k, e)


def test_autograd_function_matches_adjoint_and_oracle_fd():
    pf = _pf()
    shape = (16, 18)
    mob = G.gaussian_mobility(4, shape, width=(2.0, 4.0))
    c0, target = G.ch_initial(7, shape), G.ch_initial(8, shape)
    mf = cu(mob).to(torch.float64).requires_grad_(True)
    kappa = torch.tensor(0.6, dtype=torch.float64, requires_grad=True)
    W = torch.tensor(1.1, dtype=torch.float64, requires_grad=True)
    M = torch.tensor(0.9, dtype=torch.float64, requires_grad=True)
    loss = pf.ch_misfit(mf, kappa, W, M, cu(c0), cu(target), 0.02, 30, ckpt_every=8)
    (2.0 * loss).backward()
    def oloss(**kw):
        a = dict(W=1.1, kappa=0.6, mob=0.9)
        a.update(kw)
        return O.Problem(shape, mob_field=mob, **a).ch_adjoint(c0, target, 0.02, 30,
                                                               want_field=False)[0]
    eps = 1e-5
    for t, key, base in ((kappa, "kappa", 0.6), (W, "W", 1.1), (M, "mob", 0.9)):
        fd = (oloss(**{key: base + eps}) - oloss(**{key: base - eps})) / (2 * eps)
        assert abs(t.grad.item() - 2 * fd) <= GRAD * abs(2 * fd), key
    _, og = O.Problem(shape, W=1.1, kappa=0.6, mob=0.9, mob_field=mob).ch_adjoint(
        c0, target, 0.02, 30)
    assert rel(mf.grad.cpu().numpy(), 2 * og["mob_field"]) <= GRAD
