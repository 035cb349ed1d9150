"""Pins of the FP64 oracle to what the paper and the mathematics fix (no GPU).

Each test checks the oracle against something other than itself: closed
forms of the Q1 operators, an independent dense assembler, finite
differences of the discrete energy, exact eigenvectors of the Neumann
operators, the analytic 1-D equilibrium interface, conservation laws and the
paper's printed polynomial (Supp. 3).
"""
import math
import os

import numpy as np
import pytest

import oracle as O
import pf_inputs as G
from tests import _dense_fem as D

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def dw(W):
    return (lambda c: W * c * c * (1 - c) ** 2,
            lambda c: 2 * W * c * (1 - c) * (1 - 2 * c))


# ---------------------------------------------------------------- lumped mass

@pytest.mark.parametrize("shape,h", [((4, 4), 1.0), ((5, 7), (0.7, 1.3)), ((3, 4, 5), (1.0, 0.5, 2.0))])
def test_lumped_mass_closed_form(shape, h):
    P = O.Problem(shape, h=h)
    m = P.lumped_mass()
    hs = (h,) * len(shape) if np.isscalar(h) else h
    vol_cell = np.prod(hs)
    expect = np.full(shape, vol_cell)
    for ax in range(len(shape)):
        sl = [slice(None)] * len(shape)
        for end in (0, -1):
            sl[ax] = end
            expect[tuple(sl)] *= 0.5
    np.testing.assert_allclose(m, expect, rtol=1e-14)
    extent = np.prod([(n - 1) * hh for n, hh in zip(reversed(shape), hs)])
    assert abs(m.sum() - extent) < 1e-12 * extent


def test_lumped_mass_is_row_sum_of_dense_consistent_mass():
    Mc, _ = D.assemble(5, 4, 0.8, 1.1)
    P = O.Problem((4, 5), h=(0.8, 1.1))
    np.testing.assert_allclose(P.lumped_mass().ravel(), Mc.sum(1), rtol=1e-13)


# ---------------------------------------------------------------- stiffness

def _K_apply(shape, h, v):
    P = O.Problem(shape, h=h, W=0.0, kappa=1.0)
    return P.residual(v)


def test_q1_stiffness_stencil_2d_closed_form():
    # 2x2 Gauss integrates grad N_a . grad N_b exactly; on squares the
    # assembled interior stencil is 8/3 at the centre, -1/3 at all 8 neighbours.
    for h in (1.0, 0.37, 64 / 63):
        v = np.zeros((5, 5))
        v[2, 2] = 1.0
        r = _K_apply((5, 5), h, v)
        exp = np.zeros((5, 5))
        exp[1:4, 1:4] = -1.0 / 3.0
        exp[2, 2] = 8.0 / 3.0
        np.testing.assert_allclose(r, exp, atol=1e-14)


def test_q1_stiffness_stencil_3d_closed_form():
    # trilinear cube stencil (h = 1): centre 8/3, face 0, edge -1/6, corner -1/12, scaled by h
    h = 0.5
    v = np.zeros((5, 5, 5))
    v[2, 2, 2] = 1.0
    r = _K_apply((5, 5, 5), h, v)
    exp = np.zeros((5, 5, 5))
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                k = abs(dx) + abs(dy) + abs(dz)
                exp[2 + dz, 2 + dy, 2 + dx] = {0: 8 / 3, 1: 0.0, 2: -1 / 6, 3: -1 / 12}[k] * h
    np.testing.assert_allclose(r, exp, atol=1e-14)


@pytest.mark.parametrize("shape", [(6, 7), (4, 5, 6)])
def test_stiffness_kills_constants_and_linears(shape):
    K1 = _K_apply(shape, 1.0, np.ones(shape))
    assert np.abs(K1).max() < 1e-13
    grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    lin = 0.3 + sum((k + 1) * 0.7 * g for k, g in enumerate(grids))
    Kl = _K_apply(shape, 1.0, lin)
    inner = tuple(slice(1, -1) for _ in shape)
    assert np.abs(Kl[inner]).max() < 1e-12


# ---------------------------------------------------------------- residual

@pytest.mark.parametrize("shape,h", [((4, 4), 1.0), ((5, 7), (0.9, 1.2))])
def test_residual_matches_dense_bruteforce(shape, h):
    ny, nx = shape
    hx, hy = (h, h) if np.isscalar(h) else h
    W, kappa = 1.3, 0.7
    u = 0.5 + 0.4 * G.random_field(11, shape)
    P = O.Problem(shape, h=(hx, hy), W=W, kappa=kappa)
    _, K = D.assemble(nx, ny, hx, hy)
    F = D.nonlinear_vector(nx, ny, hx, hy, u, dw(W)[1])
    expect = F + kappa * K @ u.astype(np.float64).ravel()
    np.testing.assert_allclose(P.residual(u).ravel(), expect, rtol=1e-12, atol=1e-13)
    E = D.energy(nx, ny, hx, hy, u, dw(W)[0], kappa)
    assert abs(P.energy(u) - E) < 1e-12 * abs(E)


def _fd_gradient(fun, U, eps=1e-6):
    U = np.asarray(U, dtype=np.float64)
    g = np.zeros_like(U)
    it = np.nditer(U, flags=["multi_index"])
    for _ in it:
        idx = it.multi_index
        Up, Um = U.copy(), U.copy()
        Up[idx] += eps
        Um[idx] -= eps
        g[idx] = (fun(Up) - fun(Um)) / (2 * eps)
    return g


@pytest.mark.parametrize("case", ["ac2d", "fanchen3d"])
def test_residual_is_gradient_of_discrete_energy(case):
    if case == "ac2d":
        P = O.Problem((4, 4), h=1.1, W=1.0, kappa=0.8)
        U = 0.5 + 0.4 * G.random_field(3, (4, 4))
    else:
        P = O.Problem((3, 4, 3), h=0.9, energy="fan_chen", nf=3, kappa=0.6)
        U = 0.5 + 0.5 * G.random_field(4, (3, 3, 4, 3))
    g = _fd_gradient(P.energy, U)
    np.testing.assert_allclose(P.residual(U), g, rtol=1e-6, atol=1e-8)


def test_uniform_fixed_points():
    P = O.Problem((6, 5), W=1.0, kappa=1.0)
    for a in (0.0, 0.5, 1.0):
        assert np.abs(P.residual(np.full((6, 5), a))).max() < 1e-15


def test_fchem_matches_supp3_printed_polynomial():
    # Supp. 3 prints f_chem(eta) = 4 eta (eta - 1)(eta - 0.5), the derivative of
    # eta^2 (1 - eta)^2.  On a uniform field the gradient term vanishes and every
    # Gauss value equals the nodal value, so r_i / m_i = f'(a).
    pts = np.loadtxt(os.path.join(GOLDEN, "supp3_fchem_points.txt"))
    P = O.Problem((4, 5), W=1.0, kappa=2.0)
    m = P.lumped_mass()
    for a in pts:
        r = P.residual(np.full((4, 5), a))
        np.testing.assert_allclose(r / m, 4 * a * (a - 1) * (a - 0.5), rtol=1e-13, atol=1e-15)


# ---------------------------------------------------------------- cosine modes

def _mode(shape, k, h):
    grids = np.meshgrid(*[np.arange(n, dtype=float) for n in shape], indexing="ij")
    v = np.ones(shape)
    cs = []
    for ax, n in enumerate(shape):
        v = v * np.cos(np.pi * k[ax] * grids[ax] / (n - 1))
        cs.append(math.cos(math.pi * k[ax] / (n - 1)))
    return v, cs


def _eig(cs, h, dim):
    # 1-D stiffness (2 - 2c)/h and consistent mass h(4 + 2c)/6 per axis, divided by the lumped h^dim
    mu = np.prod([(4 + 2 * c) / 6 for c in cs])
    lam = 0.0
    for d in range(dim):
        t = (2 - 2 * cs[d]) / (h * h)
        for e in range(dim):
            if e != d:
                t *= (4 + 2 * cs[e]) / 6
        lam += t
    return mu, lam


@pytest.mark.parametrize("phi0,k", [(0.5, (3, 2)), (0.0, (1, 5)), (1.0, (4, 4))])
def test_ac_cosine_mode_growth_factor(phi0, k):
    shape, h, W, kappa, L, dt, eps = (17, 13), 0.8, 1.0, 0.6, 1.3, 0.01, 1e-6
    v, cs = _mode(shape, k, h)
    P = O.Problem(shape, h=h, W=W, kappa=kappa, mob=L)
    out = P.ac_explicit(phi0 + eps * v, dt, 1)
    mu, lam = _eig(cs, h, 2)
    fpp = 2 * W * (1 - 6 * phi0 + 6 * phi0 ** 2)
    g = 1 - dt * L * (fpp * mu + kappa * lam)
    np.testing.assert_allclose((out - phi0) / eps, g * v, atol=1e-7)


@pytest.mark.parametrize("c0,k", [(0.5, (2, 3)), (0.5, (7, 1)), (0.0, (3, 3))])
def test_ch_cosine_mode_growth_factor(c0, k):
    shape, h, W, kappa, M, dt, eps = (15, 18), 1.0, 1.0, 0.5, 1.2, 1e-3, 1e-6
    v, cs = _mode(shape, k, h)
    P = O.Problem(shape, h=h, W=W, kappa=kappa, mob=M)
    out = P.ch_explicit(c0 + eps * v, dt, 1)
    mu, lam = _eig(cs, h, 2)
    fpp = 2 * W * (1 - 6 * c0 + 6 * c0 ** 2)
    g = 1 - dt * M * lam * (fpp * mu + kappa * lam)
    np.testing.assert_allclose((out - c0) / eps, g * v, atol=1e-7)


def test_fanchen_3d_jvp_on_cosine_mode():
    # at eta = (1, 0, 0) the Fan-Chen Hessian is diagonal: 2 and -alpha + 2 gamma
    shape, h, dt, kappa, L = (5, 6, 7), 1.0, 0.5, 1.0, 1.0
    P = O.Problem(shape, h=h, energy="fan_chen", nf=3, kappa=kappa, mob=L,
                  alpha=1.0, beta=1.0, gamma=1.5)
    U = np.zeros((3,) + shape)
    U[0] = 1.0
    v, cs = _mode(shape, (1, 2, 3), h)
    V = np.zeros_like(U)
    V[2] = v
    Jv = P.implicit_jvp(dt, U, V)
    mu, lam = _eig(cs, h, 3)
    m = P.lumped_mass()
    hjj = -1.0 + 2 * 1.5
    np.testing.assert_allclose(Jv[2] / m, (1 / dt + L * (hjj * mu + kappa * lam)) * v, atol=1e-12)
    assert np.abs(Jv[:2]).max() < 1e-13


# ---------------------------------------------------------------- equilibrium interface

def test_tanh_equilibrium_profile_width_and_energy():
    # 1-D flat interface on a strip: phi -> (1 + tanh((x - x0)/delta))/2,
    # delta = sqrt(2 kappa / W); sigma = sqrt(kappa W) / (3 sqrt 2).
    W, kappa, h = 1.0, 32.0, 1.0
    delta = math.sqrt(2 * kappa / W)
    nx, ny = 257, 2
    x = np.arange(nx) * h
    x0 = x[nx // 2]
    phi = np.tile(0.5 * (1 + np.tanh((x - x0) / (0.5 * delta))), (ny, 1))
    P = O.Problem((ny, nx), h=h, W=W, kappa=kappa, mob=1.0)
    dt = 0.5 * 2 / (4 * kappa / h ** 2 + 2 * W)
    phi = P.ac_explicit(phi, dt, 3000)
    ana = 0.5 * (1 + np.tanh((x - x0) / delta))
    assert np.abs(phi[0] - ana).max() < (h / delta) ** 2
    prof = phi[0]
    lo = np.interp(0.1, prof, x)
    hi = np.interp(0.9, prof, x)
    width = 2 * delta * math.atanh(0.8)
    assert abs((hi - lo) - width) < 0.02 * width
    sigma = math.sqrt(kappa * W) / (3 * math.sqrt(2))
    assert abs(P.energy(phi) / ((ny - 1) * h) - sigma) < 0.01 * sigma


# ---------------------------------------------------------------- conservation / dissipation

@pytest.mark.parametrize("shape,h", [((5, 7), (0.7, 1.3)), ((6, 4), (1.25, 0.6)), ((4, 4), 1.0)])
def test_mobility_stiffness_matches_dense_assembly_with_field(shape, h):
    # Eq. 9 with a per-node mobility: M(x_q) = M * sum_a N_a(x_q) m_a at every
    # Gauss point.  Evaluating m at the nodes or averaging it per element would
    # give a different K_M, so a random positive field on anisotropic cells
    # separates the readings.
    ny, nx = shape
    hx, hy = (h, h) if np.isscalar(h) else h
    rng = np.random.default_rng(11 + nx * ny)
    mfield = rng.uniform(0.3, 2.5, size=shape)
    mu = rng.standard_normal(shape)
    M = 0.85
    KM = D.mobility_stiffness(nx, ny, hx, hy, mfield, M)
    P = O.Problem(shape, h=(hx, hy), mob=M, mob_field=mfield)
    got = P.mobility_stiffness_apply(mu)
    np.testing.assert_allclose(got.ravel(), KM @ mu.ravel(), rtol=0, atol=1e-13 * np.abs(KM).sum())
    # the element-averaged and node-sampled readings are far from it
    Mc, K = D.assemble(nx, ny, hx, hy)
    assert np.abs(KM @ mu.ravel() - M * mfield.ravel() * (K @ mu.ravel())).max() > 1e-3


def test_ch_step_with_mobility_field_matches_dense_assembly():
    # one explicit split-CH step, c1 = c0 - dt m^-1 K_M m^-1 (F(c0) + kappa K c0),
    # assembled from dense matrices and the dense nonlinear vector
    ny, nx, hx, hy = 5, 6, 0.9, 1.2
    rng = np.random.default_rng(5)
    mfield = rng.uniform(0.5, 1.8, size=(ny, nx))
    c0 = 0.5 + 0.2 * rng.standard_normal((ny, nx))
    W, kappa, M, dt = 1.3, 0.7, 0.9, 0.01
    _, K = D.assemble(nx, ny, hx, hy)
    KM = D.mobility_stiffness(nx, ny, hx, hy, mfield, M)
    Mc, _ = D.assemble(nx, ny, hx, hy)
    mL = Mc.sum(1)
    F = D.nonlinear_vector(nx, ny, hx, hy, c0, dw(W)[1])
    mu = (F + kappa * K @ c0.ravel()) / mL
    expect = c0.ravel() - dt * (KM @ mu) / mL
    P = O.Problem((ny, nx), h=(hx, hy), W=W, kappa=kappa, mob=M, mob_field=mfield)
    np.testing.assert_allclose(P.ch_explicit(c0, dt, 1).ravel(), expect, rtol=0, atol=1e-13)


def test_ch_mass_conserved_exactly_with_mobility_field():
    shape = (24, 20)
    mob = G.gaussian_mobility(2, shape, h=1.0, width=(2.0, 6.0))
    P = O.Problem(shape, W=1.0, kappa=0.5, mob=1.0, mob_field=mob)
    c = G.ch_initial(5, shape)
    m0 = P.mass_integral(c)
    c1 = P.ch_explicit(c, 1e-2, 300)
    assert abs(P.mass_integral(c1) - m0) < 1e-13 * abs(m0)
    assert np.abs(c1 - c).max() > 1e-3  # it did evolve


@pytest.mark.parametrize("model", ["ac", "ch"])
def test_energy_non_increasing(model):
    shape = (20, 22)
    if model == "ac":
        P = O.Problem(shape, W=1.0, kappa=1.0, mob=1.0)
        U = G.ac_initial(7, shape, 0.2, 0.8)
        step = lambda u: P.ac_explicit(u, 0.05, 1)
    else:
        P = O.Problem(shape, W=1.0, kappa=0.5, mob=1.0)
        U = G.ch_initial(7, shape)
        step = lambda u: P.ch_explicit(u, 0.02, 1)
    E = [P.energy(U)]
    for _ in range(60):
        U = step(U)
        E.append(P.energy(U))
    d = np.diff(E)
    assert (d <= 1e-14 * abs(E[0])).all()
    assert E[-1] < E[0]


# ---------------------------------------------------------------- implicit: JVP, GMRES, Newton

@pytest.mark.parametrize("case", ["ac2d", "fanchen3d"])
def test_jvp_matches_fd_of_residual_and_is_symmetric(case):
    dt = 0.5
    if case == "ac2d":
        shape, P = (6, 7), O.Problem((6, 7), W=1.0, kappa=0.8, mob=1.2)
        U = 0.5 + 0.4 * G.random_field(1, shape)
        v = G.random_field(2, shape)
        w = G.random_field(3, shape)
    else:
        shape = (3, 4, 5, 4)
        P = O.Problem(shape[1:], energy="fan_chen", nf=3, kappa=1.0, mob=1.0)
        U = 0.5 + 0.5 * G.random_field(1, shape)
        v = G.random_field(2, shape)
        w = G.random_field(3, shape)
    U, v, w = (a.astype(np.float64) for a in (U, v, w))
    Un = np.zeros_like(U)
    eps = 1e-6
    fd = (P.implicit_residual(dt, Un, U + eps * v) - P.implicit_residual(dt, Un, U - eps * v)) / (2 * eps)
    Jv = P.implicit_jvp(dt, U, v)
    np.testing.assert_allclose(Jv, fd, rtol=1e-6, atol=1e-8)
    Jw = P.implicit_jvp(dt, U, w)
    assert abs(np.vdot(w, Jv) - np.vdot(v, Jw)) < 1e-12 * np.abs(Jv).sum()


def test_gmres_recovers_known_solution():
    shape = (3, 6, 5, 4)
    P = O.Problem(shape[1:], energy="fan_chen", nf=3, kappa=1.0, mob=1.0)
    U = 0.5 + 0.5 * G.random_field(8, shape)
    xs = G.random_field(9, shape).astype(np.float64)
    b = P.implicit_jvp(0.5, U, xs)
    x, ok, it = P.gmres(0.5, U, b, restart=20, rtol=1e-12)
    assert ok
    np.testing.assert_allclose(x, xs, atol=1e-9)


def test_newton_root_reevaluated():
    shape = (3, 8, 7, 6)
    P = O.Problem(shape[1:], energy="fan_chen", nf=3, kappa=1.0, mob=1.0)
    Un = np.clip(0.5 + 0.6 * G.random_field(5, shape), 0, 1).astype(np.float64)
    U, st = P.newton(0.5, Un, abs_tol=1e-11)
    assert st["ok"] and st["newton_iters"] >= 2
    R = P.implicit_residual(0.5, Un, U)
    assert np.linalg.norm(R) <= 1e-11
    # the implicit step dissipates energy: E(U^{n+1}) <= E(U^n)
    assert P.energy(U) <= P.energy(Un)


# ---------------------------------------------------------------- adjoint

def _adj_problem(mob_field=None, **kw):
    shape = (12, 10)
    base = dict(W=1.0, kappa=0.5, mob=1.0)
    base.update(kw)
    return O.Problem(shape, mob_field=mob_field, **base), shape


def test_adjoint_matches_central_fd_scalars_and_mobility_field():
    shape = (12, 10)
    mob = G.gaussian_mobility(3, shape, h=1.0, width=(2.0, 5.0)).astype(np.float64)
    c0 = G.ch_initial(4, shape).astype(np.float64)
    target = G.ch_initial(5, shape).astype(np.float64)
    dt, N = 0.02, 25
    P, _ = _adj_problem(mob, W=1.1, kappa=0.6, mob=0.9)
    loss, g = P.ch_adjoint(c0, target, dt, N)

    def L(**kw):
        args = dict(W=1.1, kappa=0.6, mob=0.9)
        mf = kw.pop("mob_field", mob)
        args.update(kw)
        Q, _ = _adj_problem(mf, **args)
        l, _ = Q.ch_adjoint(c0, target, dt, N, want_field=False)
        return l

    eps = 1e-5
    for name, key, base in (("kappa", "kappa", 0.6), ("W", "W", 1.1), ("M", "mob", 0.9)):
        fd = (L(**{key: base + eps}) - L(**{key: base - eps})) / (2 * eps)
        assert abs(g[name] - fd) <= 1e-6 * max(1.0, abs(fd)), (name, g[name], fd)
    d = G.gaussian_mobility(9, shape, h=1.0, width=(2.0, 5.0)).astype(np.float64) - 1.0
    fd = (L(mob_field=mob + eps * d) - L(mob_field=mob - eps * d)) / (2 * eps)
    assert abs(np.vdot(g["mob_field"], d) - fd) <= 1e-6 * max(1e-3, abs(fd))
    for node in [(0, 0), (5, 4), (11, 9), (3, 0)]:
        e = np.zeros(shape)
        e[node] = 1.0
        fd = (L(mob_field=mob + eps * e) - L(mob_field=mob - eps * e)) / (2 * eps)
        assert abs(g["mob_field"][node] - fd) <= 1e-6 * max(1e-4, abs(fd)), node


def test_adjoint_one_step_dot_product():
    # <lambda, G'(c) v> == <G'(c)^T lambda, v>; G' v by central FD of one forward step.
    shape = (9, 11)
    mob = G.gaussian_mobility(6, shape, width=(2.0, 4.0)).astype(np.float64)
    P = O.Problem(shape, W=1.0, kappa=0.5, mob=1.0, mob_field=mob)
    c = G.ch_initial(1, shape).astype(np.float64)
    lam = G.random_field(2, shape).astype(np.float64)
    v = G.random_field(3, shape).astype(np.float64)
    dt = 0.05
    c1 = P.ch_explicit(c, dt, 1)
    # nodal loss 1/2 |c1 - target|^2 with target = c1 - lam gives lambda^1 = lam
    _, g = P.ch_adjoint(c, c1 - lam, dt, 1, nodal_loss=True, want_field=False)
    eps = 1e-6
    Gv = (P.ch_explicit(c + eps * v, dt, 1) - P.ch_explicit(c - eps * v, dt, 1)) / (2 * eps)
    assert abs(np.vdot(lam, Gv) - np.vdot(g["c0"], v)) < 1e-8 * np.abs(lam * Gv).sum()
