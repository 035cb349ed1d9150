"""Pins of the oracle's implicit split Cahn-Hilliard step (Eq. 9-10 with
backward Euler, Eq. 13; unknowns [c, mu]): the Jacobian action against central
finite differences of the residual, exact conservation of c at the Newton
root, consistency with the explicit step as dt -> 0 (first-order schemes that
agree to O(dt^2) per step), energy decrease, and the refactored gradient-flow
Newton still reaching its root."""
import numpy as np

import oracle as O
import pf_inputs as G


def problem(shape=(9, 11), h=(1.0, 1.1)):
    return O.Problem(shape, h=h, W=1.0, kappa=0.5, mob=1.0)


def test_jvp_is_the_derivative_of_the_residual():
    P = problem()
    rng = np.random.default_rng(3)
    cn = 0.5 + 0.05 * rng.standard_normal(P.shape)
    U = np.stack([cn + 0.01 * rng.standard_normal(P.shape), rng.standard_normal(P.shape)])
    v = rng.standard_normal(U.shape)
    eps = 1e-6
    fd = (P.chsplit_residual(0.1, cn, U + eps * v) - P.chsplit_residual(0.1, cn, U - eps * v)) / (
        2 * eps)
    jv = P.chsplit_jvp(0.1, U, v)
    assert np.abs(jv - fd).max() <= 1e-7 * np.abs(fd).max()


def test_implicit_step_conserves_c_and_decreases_energy():
    shape = (33, 29)
    P = problem(shape, 1.0)
    c = G.ch_initial(4, shape).astype(np.float64)
    m0, E0 = P.mass_integral(c), P.energy(c)
    for _ in range(3):
        U, info = P.chsplit_newton(0.05, c, abs_tol=1e-11)
        assert info["ok"]
        c = U[0]
    assert abs(P.mass_integral(c) - m0) <= 1e-12 * abs(m0)
    assert P.energy(c) < E0
    # the root's second block is the chemical potential of its first
    assert np.abs(U[1] - P.chemical_potential(U[0])).max() <= 1e-8


def test_implicit_and_explicit_steps_agree_to_second_order_in_dt():
    shape = (17, 19)
    P = problem(shape, 1.0)
    c = G.ch_initial(5, shape).astype(np.float64)
    diffs = []
    for dt in (2e-3, 1e-3):
        U, info = P.chsplit_newton(dt, c, abs_tol=1e-9)
        assert info["ok"]
        diffs.append(np.abs(U[0] - P.ch_explicit(c, dt, 1)).max())
    ratio = diffs[0] / diffs[1]
    assert 3.5 < ratio < 4.5, ratio


def test_gradient_flow_newton_reaches_its_root():
    shape = (9, 8)
    P = O.Problem(shape, W=1.0, kappa=1.0, mob=1.0)
    Un = G.ac_initial(2, shape, 0.2, 0.8).astype(np.float64)
    U, info = P.newton(0.5, Un, abs_tol=1e-12)
    assert info["ok"]
    assert np.linalg.norm(P.implicit_residual(0.5, Un, U)) <= 1e-12


def test_implicit_adjoint_sensitivities_match_central_differences():
    # Table 1 setting: a 64 x 64 mesh on a domain of 100 x 100, objective the
    # domain average of the order parameter (Eq. 19), theta = (L, kappa); dt L
    # max|f''| < 1 keeps every implicit step's root unique (so O is smooth in theta)
    shape, h = (64, 64), 100.0 / 63.0
    U0 = G.ac_initial(11, shape, 0.2, 0.8).astype(np.float64)

    def obj(L, kappa):
        P = O.Problem(shape, h=h, W=1.0, kappa=kappa, mob=L)
        return P.implicit_adjoint(U0, 0.5, 6)

    O0, g = obj(1.0, 2.0)
    eps = 1e-5
    fd = [(obj(1.0 + eps, 2.0)[0] - obj(1.0 - eps, 2.0)[0]) / (2 * eps),
          (obj(1.0, 2.0 + eps)[0] - obj(1.0, 2.0 - eps)[0]) / (2 * eps)]
    for a, b in zip(g, fd):
        assert abs(a - b) <= 1e-6 * max(abs(b), 1e-3), (g, fd)


def test_implicit_adjoint_3d_fan_chen_matches_central_differences():
    # the same reverse sweep on the 3-D grain-growth (Fan-Chen) operators: a
    # 7 x 6 x 5 node mesh with 3 order parameters, Voronoi-like start, theta =
    # (L, kappa); FP64 central differences of the oracle's own forward solve
    shape = (5, 6, 7)
    rng = np.random.default_rng(3)
    U0 = np.clip(rng.uniform(-0.2, 1.2, size=(3,) + shape), 0.0, 1.0)

    def obj(L, kappa):
        P = O.Problem(shape, energy="fan_chen", nf=3, kappa=kappa, mob=L, alpha=1.0, beta=1.0,
                      gamma=1.5)
        return P.implicit_adjoint(U0, 0.5, 3)

    O0, g = obj(1.0, 1.0)
    eps = 1e-5
    fd = [(obj(1.0 + eps, 1.0)[0] - obj(1.0 - eps, 1.0)[0]) / (2 * eps),
          (obj(1.0, 1.0 + eps)[0] - obj(1.0, 1.0 - eps)[0]) / (2 * eps)]
    for a, b in zip(g, fd):
        assert abs(a - b) <= 1e-6 * max(abs(b), 1e-3), (g, fd)
    assert min(abs(v) for v in fd) > 1e-4  # both sensitivities are non-trivial here
