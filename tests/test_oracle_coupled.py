"""Pins of the oracle's coupled Allen-Cahn / Cahn-Hilliard model (Eq. 7 with
the Supp. 3 polynomials; explicit Euler of Eq. 9-12): the energy of uniform
states against the printed polynomials, residual and Hessian against central
finite differences, exact conservation of c, uniform fixed points and the
monotone decrease of the discrete energy."""
import os

import numpy as np

import oracle as O
import pf_inputs as G

HERE = os.path.dirname(os.path.abspath(__file__))


def printed():
    coef = {}
    for line in open(os.path.join(HERE, "golden", "supp3_coupled_polynomials.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        coef[name] = [float(v) for v in vals]
    return coef


def peval(a, x):
    return sum(ak * x ** k for k, ak in enumerate(a))


def problem(shape=(5, 6), h=(0.7, 1.3)):
    return O.Problem(shape, h=h, energy="coupled", kappa=0.3, mob=1.0, mob2=150.0)


def test_uniform_state_energy_is_the_printed_polynomials():
    co = printed()
    P = problem()
    area = (6 - 1) * 0.7 * (5 - 1) * 1.3
    for c0, e0 in [(0.2, 0.0), (0.6, 1.0), (0.45, 0.3), (0.9, 0.75)]:
        U = np.stack([np.full((5, 6), c0), np.full((5, 6), e0)])
        hh = peval(co["h"], e0)
        f = peval(co["f_alpha"], c0) * (1 - hh) + peval(co["f_beta"], c0) * hh
        assert abs(P.energy(U) - area * f) <= 1e-12 * abs(area * f)


def test_residual_is_the_gradient_of_the_energy():
    P = problem((4, 5), (0.9, 1.1))
    rng = np.random.default_rng(1)
    U = np.stack([0.6 + 0.1 * rng.standard_normal((4, 5)), rng.uniform(0, 1, (4, 5))])
    r = P.residual(U)
    eps = 1e-6
    fd = np.zeros_like(U)
    for idx in np.ndindex(U.shape):
        Up, Um = U.copy(), U.copy()
        Up[idx] += eps
        Um[idx] -= eps
        fd[idx] = (P.energy(Up) - P.energy(Um)) / (2 * eps)
    assert np.abs(r - fd).max() <= 1e-7 * np.abs(fd).max()
    # the c residual carries no gradient term: a c field alone in one node moves
    # only through the local energy
    assert np.abs(r[0]).max() > 0 and np.abs(r[1]).max() > 0


def test_hessian_is_the_derivative_of_the_residual():
    P = problem((4, 5), (1.0, 1.0))
    rng = np.random.default_rng(2)
    U = np.stack([0.6 + 0.1 * rng.standard_normal((4, 5)), rng.uniform(0, 1, (4, 5))])
    v = rng.standard_normal(U.shape)
    eps = 1e-6
    fd = (P.residual(U + eps * v) - P.residual(U - eps * v)) / (2 * eps)
    hv = P.hessian_apply(U, v)
    assert np.abs(hv - fd).max() <= 1e-7 * np.abs(fd).max()


def test_explicit_step_conserves_c_and_decreases_the_energy():
    shape = (33, 41)
    U0 = G.coupled_initial(3, shape).astype(np.float64)
    P = O.Problem(shape, energy="coupled", kappa=0.3, mob=1.0, mob2=150.0)
    m0 = P.mass_integral(U0[0])
    E = [P.energy(U0)]
    U = U0
    for _ in range(6):
        U = P.coupled_explicit(U, 1e-3, 20)
        E.append(P.energy(U))
    assert abs(P.mass_integral(U[0]) - m0) <= 1e-13 * abs(m0)
    assert all(b < a for a, b in zip(E, E[1:]))
    assert np.abs(U[1] - U0[1]).max() > 1e-3  # eta moved


def test_uniform_states_with_eta_zero_or_one_are_fixed_points():
    shape = (7, 9)
    P = O.Problem(shape, energy="coupled", kappa=0.3, mob=1.0, mob2=150.0)
    for c0, e0 in [(0.3, 0.0), (0.7, 1.0)]:
        U = np.stack([np.full(shape, c0), np.full(shape, e0)])
        out = P.coupled_explicit(U, 1e-3, 10)
        assert np.abs(out - U).max() <= 1e-14
