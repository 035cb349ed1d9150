"""GPU parity of the 3-D implicit operators and the Newton-GMRES step vs the oracle.

The JVP and residual (Eq. 14) are compared element by element with the FP64
oracle; the Newton root is compared with the oracle's FP64 Newton root (tight
tolerances on both sides, so the difference is the FP32 noise floor); at the
grain-growth size (128^3, 8 order parameters) the GPU root is re-evaluated by
the oracle's FP64 residual, a property that holds at any size.
"""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu

FC = dict(alpha=1.0, beta=1.0, gamma=1.5)


def _pf():
    import paper_2601_06079_gb300 as pf
    return pf


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def solver3d(shape, nf, model="fanchen", h=1.0, kappa=1.0, mob=1.0, dt=0.5, W=1.0):
    pf = _pf()
    s = pf.Solver(shape, h=h, model=model, n_fields=nf)
    s.set_params(W=W, kappa=kappa, mobility=mob, dt=dt, shift=0.0, **FC)
    return s


def oracle3d(shape, nf, model="fanchen", h=1.0, kappa=1.0, mob=1.0, W=1.0):
    return O.Problem(shape, h=h, energy="fan_chen" if model == "fanchen" else "double_well",
                     nf=nf, kappa=kappa, mob=mob, W=W, **FC)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape,nf,h", [((5, 6, 7), 1, 1.0), ((9, 10, 11), 3, 0.8),
                                        ((17, 9, 12), 8, 1.0), ((3, 2, 4), 2, (1.0, 0.7, 1.3))])
def test_jvp_and_residual_match_oracle(shape, nf, h):
    s = solver3d(shape, nf, h=h, kappa=0.9, mob=1.1)
    P = oracle3d(shape, nf, h=h, kappa=0.9, mob=1.1)
    U = G.random_field(1, (nf,) + shape, 0.0, 1.0)
    Un = G.random_field(2, (nf,) + shape, 0.0, 1.0)
    v = G.random_field(3, (nf,) + shape)
    if nf == 1:
        U, Un, v = U[0], Un[0], v[0]
    Jv = s.jvp(cu(U), cu(v)).cpu().numpy()
    ref = P.implicit_jvp(0.5, U, v)
    assert rel(Jv, ref) <= 2e-6
    R = s.implicit_residual(cu(Un), cu(U)).cpu().numpy()
    ref = P.implicit_residual(0.5, Un, U)
    assert rel(R, ref) <= 2e-6


def test_double_well_3d_jvp_matches_oracle():
    shape = (8, 9, 10)
    s = solver3d(shape, 1, model="ac", kappa=0.7, mob=1.3, W=1.2)
    P = oracle3d(shape, 1, model="ac", kappa=0.7, mob=1.3, W=1.2)
    U = G.random_field(4, shape, 0.0, 1.0)
    v = G.random_field(5, shape)
    assert rel(s.jvp(cu(U), cu(v)).cpu().numpy(), P.implicit_jvp(0.5, U, v)) <= 2e-6


@pytest.mark.parametrize("shape,nf", [((12, 10, 9), 4), ((9, 17, 8), 8)])
def test_newton_root_matches_oracle(shape, nf):
    U0 = np.clip(0.5 + 0.6 * G.random_field(7, (nf,) + shape), 0, 1).astype(np.float32)
    s = solver3d(shape, nf)
    t = cu(U0)
    st = s.step_implicit(t, 1, newton_rtol=1e-6, gmres_rtol=1e-4)
    assert st["converged"] and st["newton_iters"] >= 2
    P = oracle3d(shape, nf)
    ref, ost = P.newton(0.5, U0, abs_tol=1e-10)
    assert ost["ok"]
    assert rel(t.cpu().numpy(), ref) <= 1e-5


def test_multi_step_implicit_matches_oracle():
    shape, nf = (10, 11, 9), 3
    U0 = np.clip(0.5 + 0.6 * G.random_field(9, (nf,) + shape), 0, 1).astype(np.float32)
    s = solver3d(shape, nf)
    t = cu(U0)
    st = s.step_implicit(t, 4, newton_rtol=1e-6, gmres_rtol=1e-4)
    assert st["converged"]
    P = oracle3d(shape, nf)
    ref = U0.astype(np.float64)
    for _ in range(4):
        ref, ost = P.newton(0.5, ref, abs_tol=1e-10)
    assert rel(t.cpu().numpy(), ref) <= 2e-5
    assert P.energy(t.cpu().numpy()) < P.energy(U0)


def test_uniform_state_needs_no_newton_iteration():
    s = solver3d((6, 7, 8), 2)
    t = torch.zeros((2, 6, 7, 8), device="cuda")
    st = s.step_implicit(t, 2)
    assert st["newton_iters"] == 0 and torch.count_nonzero(t) == 0


def test_explicit_3d_matches_oracle():
    shape, nf = (7, 9, 8), 2
    U0 = G.random_field(3, (nf,) + shape, 0.0, 1.0)
    s = solver3d(shape, nf, dt=0.02)
    t = cu(U0)
    s.step_explicit(t, 25)
    ref = oracle3d(shape, nf).ac_explicit(U0, 0.02, 25)
    assert rel(t.cpu().numpy(), ref) <= 1e-5


def test_grain_growth_128_cubed_root_reevaluated_by_oracle():
    # 128^3 nodes, 8 Fan-Chen order parameters (Voronoi start), dt = 0.5
    U0 = G.voronoi_grains(1, n=128, n_seeds=64, n_op=8)
    s = solver3d((128, 128, 128), 8)
    t = cu(U0)
    st = s.step_implicit(t, 1)
    assert st["converged"]
    P = oracle3d((128, 128, 128), 8)
    R = P.implicit_residual(0.5, U0, t.cpu().numpy())
    ref = np.linalg.norm(P.lumped_mass()[None] * U0.astype(np.float64) / 0.5)
    assert np.linalg.norm(R) <= 2e-5 * ref


# ---------------------------------------------------------------- 2-D Allen-Cahn


def _ac2d(shape, h, W=1.3, kappa=0.7, L=1.1, dt=0.5):
    import paper_2601_06079_gb300 as pf
    s = pf.Solver(shape, h=h, model="ac")
    s.set_params(W=W, kappa=kappa, mobility=L, dt=dt)
    P = O.Problem(shape, h=h, energy="double_well", W=W, kappa=kappa, mob=L)
    return s, P


@pytest.mark.parametrize("shape,h", [((37, 45), 1.0), ((64, 130), (0.9, 1.2)), ((3, 5), 1.0)])
def test_2d_jvp_and_residual_match_oracle(shape, h):
    s, P = _ac2d(shape, h)
    U = G.ac_initial(3, shape, 0.2, 0.8)
    Un = G.ac_initial(4, shape, 0.2, 0.8)
    v = G.random_field(5, shape)
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    assert rel(s.jvp(cu(U), cu(v)).cpu().numpy(), P.implicit_jvp(0.5, U, v)) <= 2e-6
    assert rel(s.implicit_residual(cu(Un), cu(U)).cpu().numpy(),
               P.implicit_residual(0.5, Un, U)) <= 2e-6


def test_2d_newton_steps_match_oracle():
    # the paper's implicit benchmarks take large steps; 4 backward-Euler steps of
    # dt = 0.5 from a noisy start on a ragged mesh
    shape = (67, 90)
    s, P = _ac2d(shape, 1.0)
    U0 = G.ac_initial(6, shape, 0.3, 0.7)
    t = torch.from_numpy(U0).cuda()
    st = s.step_implicit(t, 4, newton_rtol=1e-6, gmres_rtol=1e-4)
    assert st["converged"]
    ref = U0.astype(np.float64)
    for _ in range(4):
        ref, info = P.newton(0.5, ref, abs_tol=1e-12, gmres_rtol=1e-10)
        assert info["ok"]
    assert rel(t.cpu().numpy(), ref) <= 2e-5


def test_2d_implicit_root_reevaluated_by_oracle_at_1024():
    shape = (1024, 1024)
    s, P = _ac2d(shape, 1.0, W=1.0, kappa=1.0, L=1.0, dt=1.0)
    U0 = G.ac_initial(7, shape)
    t = torch.from_numpy(U0).cuda()
    st = s.step_implicit(t, 1)
    assert st["converged"] and st["newton_iters"] >= 1
    R = P.implicit_residual(1.0, U0.astype(np.float64), t.cpu().numpy().astype(np.float64))
    m = P.lumped_mass()
    ref = np.linalg.norm(m * U0.astype(np.float64) / 1.0)
    assert np.linalg.norm(R) <= 2e-5 * ref


# ---------------------------------------------------------------- 2-D split Cahn-Hilliard


def _ch2d(shape, h, dt=0.05):
    import paper_2601_06079_gb300 as pf
    s = pf.Solver(shape, h=h, model="ch")
    s.set_params(W=1.0, kappa=0.5, mobility=1.0, dt=dt)
    P = O.Problem(shape, h=h, W=1.0, kappa=0.5, mob=1.0)
    return s, P


@pytest.mark.parametrize("shape,h", [((37, 45), 1.0), ((64, 130), (0.9, 1.2)), ((3, 4), 1.0)])
def test_2d_ch_split_jvp_and_residual_match_oracle(shape, h):
    s, P = _ch2d(shape, h)
    cn = G.ch_initial(3, shape)
    U = np.stack([G.ch_initial(4, shape), G.random_field(5, shape)])
    v = np.stack([G.random_field(6, shape), G.random_field(7, shape)])
    Un = np.stack([cn, np.zeros(shape, np.float32)])
    cu = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    assert rel(s.jvp(cu(U), cu(v)).cpu().numpy(), P.chsplit_jvp(0.05, U, v)) <= 2e-6
    assert rel(s.implicit_residual(cu(Un), cu(U)).cpu().numpy(),
               P.chsplit_residual(0.05, cn, U)) <= 2e-6


def test_2d_ch_implicit_steps_match_oracle_and_conserve_c():
    shape = (67, 90)
    s, P = _ch2d(shape, 1.0, dt=0.05)
    c0 = G.ch_initial(8, shape)
    t = torch.from_numpy(c0).cuda()
    st = s.step_implicit(t, 3, newton_rtol=1e-7, gmres_rtol=1e-5)
    assert st["converged"]
    ref = c0.astype(np.float64)
    for _ in range(3):
        U, info = P.chsplit_newton(0.05, ref, abs_tol=1e-9)
        assert info["ok"]
        ref = U[0]
    got = t.cpu().numpy()
    assert rel(got, ref) <= 1e-5
    m0 = P.mass_integral(c0.astype(np.float64))
    assert abs(P.mass_integral(got.astype(np.float64)) - m0) <= 1e-6 * abs(m0)


def test_2d_ch_implicit_large_step_1024():
    # a step 1000x the explicit one of the bench (dt 1e-3), as the paper's
    # implicit benchmarks take: Newton converges and c is conserved
    shape = (1024, 1024)
    s, P = _ch2d(shape, 1.0, dt=1.0)
    c0 = G.ch_initial(9, shape)
    t = torch.from_numpy(c0).cuda()
    st = s.step_implicit(t, 2)
    assert st["converged"] and st["newton_iters"] >= 2
    m0 = P.mass_integral(c0.astype(np.float64))
    assert abs(P.mass_integral(t.cpu().numpy().astype(np.float64)) - m0) <= 1e-6 * abs(m0)


# ---------------------------------------------------------------- implicit adjoint


def test_implicit_adjoint_matches_oracle_table1_setting():
    # Table 1 setting: 64 x 64 mesh on a 100 x 100 domain, objective the domain
    # average of eta (Eq. 19), theta = (L, kappa); bar 0.1 per mille
    import paper_2601_06079_gb300 as pf
    shape, h = (64, 64), 100.0 / 63.0
    U0 = G.ac_initial(11, shape, 0.2, 0.8)
    s = pf.Solver(shape, h=h, model="ac")
    s.set_params(W=1.0, kappa=2.0, mobility=1.0, dt=0.5)
    # adjoint solves to 1e-7 (FP32 Newton itself stops near 1e-7 relative)
    O_gpu, g, st = s.implicit_adjoint(torch.from_numpy(U0).cuda(), 6, newton_rtol=1e-7,
                                      gmres_rtol=1e-7)
    P = O.Problem(shape, h=h, W=1.0, kappa=2.0, mob=1.0)
    O_ref, g_ref = P.implicit_adjoint(U0.astype(np.float64), 0.5, 6)
    assert abs(O_gpu - O_ref) <= 1e-6 * abs(O_ref)
    print("Table 1 setting rel errors (L, kappa):", abs(g["L"] - g_ref[0]) / abs(g_ref[0]),
          abs(g["kappa"] - g_ref[1]) / abs(g_ref[1]))
    assert abs(g["L"] - g_ref[0]) <= 1e-4 * abs(g_ref[0]), (g, g_ref)
    assert abs(g["kappa"] - g_ref[1]) <= 1e-4 * abs(g_ref[1]), (g, g_ref)


def test_implicit_adjoint_3d_fan_chen_matches_oracle_adjoint():
    # the same reverse sweep on the 3-D grain-growth operators (symmetric J),
    # against the oracle's discrete adjoint (pinned to FP64 central differences
    # on the CPU): 16^3 nodes, 4 order parameters, 3 steps of dt = 0.5
    import paper_2601_06079_gb300 as pf
    from paper_2601_06079_gb300 import warmstart as WS
    n = 16
    U0 = G.voronoi_grains(3, n=n, n_seeds=6, n_op=4)
    s = pf.Solver((n, n, n), model="fanchen", n_fields=4)
    s.set_params(dt=0.5, **{**WS.FANCHEN, "mobility": 1.0, "kappa": 1.0})
    O_gpu, g, _ = s.implicit_adjoint(torch.from_numpy(U0).cuda(), 3, newton_rtol=1e-7,
                                     gmres_rtol=1e-6)
    fc = WS.FANCHEN
    P = O.Problem((n, n, n), energy="fan_chen", nf=4, kappa=1.0, mob=1.0, alpha=fc["alpha"],
                  beta=fc["beta"], gamma=fc["gamma"])
    O_ref, g_ref = P.implicit_adjoint(U0.astype(np.float64), 0.5, 3)
    errs = (abs(O_gpu - O_ref) / abs(O_ref), abs(g["L"] - g_ref[0]) / abs(g_ref[0]),
            abs(g["kappa"] - g_ref[1]) / abs(g_ref[1]))
    print("3-D Fan-Chen implicit adjoint rel errors (O, L, kappa):", errs)
    assert errs[0] <= 1e-6
    assert errs[1] <= 1e-4, (g, g_ref)
    assert errs[2] <= 1e-4, (g, g_ref)


def test_workspace_growth_between_explicit_and_implicit_steps():
    # a Solver binds the explicit part of its workspace first; the first
    # implicit step grows it (dropping the captured explicit-step graph), and
    # explicit steps on the new memory continue the same trajectory
    shape = (67, 90)
    s, P = _ac2d(shape, 1.0)
    small = s._ws.numel()
    U0 = G.ac_initial(11, shape, 0.3, 0.7)
    t = torch.from_numpy(U0).cuda()
    s.set_params(W=1.3, kappa=0.7, mobility=1.1, dt=0.01)
    s.step_explicit(t, 130)  # two 64-step graph replays and two single steps
    s.set_params(W=1.3, kappa=0.7, mobility=1.1, dt=0.5)
    st = s.step_implicit(t, 1, newton_rtol=1e-6, gmres_rtol=1e-4)
    assert st["converged"] and s._ws.numel() > small
    s.set_params(W=1.3, kappa=0.7, mobility=1.1, dt=0.01)
    s.step_explicit(t, 130)
    ref = P.ac_explicit(U0, 0.01, 130)
    ref, info = P.newton(0.5, ref, abs_tol=1e-12, gmres_rtol=1e-10)
    assert info["ok"]
    ref = P.ac_explicit(ref, 0.01, 130)
    assert rel(t.cpu().numpy(), ref) <= 2e-5
