"""Pins of the FP64 Eshelby-inclusion oracle (Eq. 3-4, Supp. 3 Eq. III.1,
objective Eq. 21-22) against facts that do not come from the oracle itself:
an independent element assembly, rigid-body and affine fields, an exact
solution, the mean-strain identity of a traction-free body, the radial
solution of a spherical inclusion, and finite differences."""
import numpy as np
import pytest

import oracle as O

E0, NU0 = 22.5, 0.3  # Supp. 3


def lame(E, nu):
    return E * nu / ((1 + nu) * (1 - 2 * nu)), E / (2 * (1 + nu))


def voigt_element_stiffness(h, lam, mu, npts=3):
    """Independent element stiffness: Voigt strains B (6 x 24, engineering
    shears), D the isotropic 6 x 6 matrix, K = sum_q w B^T D B with an npts-point
    Gauss-Legendre rule per axis (3 points integrate the degree-4 integrand
    exactly as 2 do).  DOFs ordered component-major over the 8 corners, like
    the oracle's global vectors on a 2x2x2 node mesh."""
    xg, wg = np.polynomial.legendre.leggauss(npts)
    xg, wg = 0.5 * (xg + 1), 0.5 * wg
    D = np.zeros((6, 6))
    D[:3, :3] = lam
    D[np.arange(3), np.arange(3)] += 2 * mu
    D[3:, 3:] = mu * np.eye(3)
    K = np.zeros((24, 24))
    for iz, (z, wz) in enumerate(zip(xg, wg)):
        for iy, (y, wy) in enumerate(zip(xg, wg)):
            for ix, (x, wx) in enumerate(zip(xg, wg)):
                B = np.zeros((6, 24))
                for a in range(8):
                    ax, ay, az = a & 1, (a >> 1) & 1, a >> 2
                    Nx, Ny, Nz = (x if ax else 1 - x), (y if ay else 1 - y), (z if az else 1 - z)
                    gx = (1 if ax else -1) / h[0] * Ny * Nz
                    gy = Nx * (1 if ay else -1) / h[1] * Nz
                    gz = Nx * Ny * (1 if az else -1) / h[2]
                    cx, cy, cz = a, 8 + a, 16 + a
                    B[0, cx], B[1, cy], B[2, cz] = gx, gy, gz
                    B[3, cx], B[3, cy] = gy, gx      # 2 eps_xy
                    B[4, cy], B[4, cz] = gz, gy      # 2 eps_yz
                    B[5, cx], B[5, cz] = gz, gx      # 2 eps_xz
                K += wx * wy * wz * h[0] * h[1] * h[2] * B.T @ D @ B
    return K


def dense_single_element(h, lam, mu):
    el = O.Elastic((2, 2, 2), h=h)
    K = np.zeros((24, 24))
    for c in range(24):
        e = np.zeros(24)
        e[c] = 1.0
        K[:, c] = el.apply(e.reshape(3, 2, 2, 2), lam, mu).ravel()
    return K


def coords(shape, h):
    nz, ny, nx = shape
    z, y, x = np.meshgrid(np.arange(nz) * h[2], np.arange(ny) * h[1], np.arange(nx) * h[0],
                          indexing="ij")
    return x, y, z


def test_lame_constants_closed_form():
    lam, mu = O.Elastic.lame(E0, NU0)
    assert lam == pytest.approx(22.5 * 0.3 / (1.3 * 0.4), rel=1e-15)
    assert mu == pytest.approx(22.5 / 2.6, rel=1e-15)


def test_element_stiffness_matches_independent_voigt_assembly():
    h = (1.0, 1.3, 0.7)
    lam, mu = lame(E0, NU0)
    K = dense_single_element(h, lam, mu)
    Kv = voigt_element_stiffness(h, lam, mu)
    assert np.abs(K - Kv).max() <= 1e-12 * np.abs(Kv).max()


def test_element_stiffness_symmetric_with_six_rigid_modes():
    h = (0.8, 1.1, 1.5)
    lam, mu = lame(E0, NU0)
    K = dense_single_element(h, lam, mu)
    assert np.abs(K - K.T).max() <= 1e-13 * np.abs(K).max()
    ev = np.linalg.eigvalsh(0.5 * (K + K.T))
    scale = ev.max()
    assert np.sum(np.abs(ev) <= 1e-12 * scale) == 6
    assert ev[6] > 1e-3 * scale
    x, y, z = coords((2, 2, 2), (h[0], h[1], h[2]))
    one, zero = np.ones_like(x), np.zeros_like(x)
    modes = [np.stack([one, zero, zero]), np.stack([zero, one, zero]), np.stack([zero, zero, one]),
             np.stack([-y, x, zero]), np.stack([zero, -z, y]), np.stack([z, zero, -x])]
    for md in modes:
        assert np.abs(K @ md.ravel()).max() <= 1e-12 * scale


def test_uniform_strain_energy_and_patch_test():
    shape, h = (4, 5, 6), (0.9, 1.2, 0.8)
    lam, mu = lame(E0, NU0)
    rng = np.random.default_rng(3)
    A = rng.standard_normal((3, 3))
    x, y, z = coords(shape, h)
    X = np.stack([x, y, z])
    u = np.einsum("ij,j...->i...", A, X)
    Ku = O.Elastic(shape, h).apply(u, lam, mu)
    eps = 0.5 * (A + A.T)
    V = (shape[2] - 1) * h[0] * (shape[1] - 1) * h[1] * (shape[0] - 1) * h[2]
    energy = V * (lam * np.trace(eps) ** 2 + 2 * mu * np.sum(eps * eps))
    assert float(np.sum(u * Ku)) == pytest.approx(energy, rel=1e-12)
    # an affine field is in equilibrium at every interior node
    assert np.abs(Ku[:, 1:-1, 1:-1, 1:-1]).max() <= 1e-12 * np.abs(Ku).max()


def test_rhs_matches_independent_voigt_quadrature():
    shape, h = (3, 4, 3), (10.0, 7.0, 9.0)
    lam, mu = lame(E0, NU0)
    m, l, a = 0.01, 0.2, 12.0
    f = O.Elastic(shape, h).rhs(lam, mu, m, l, a)
    nz, ny, nx = shape
    ref = np.zeros((3,) + shape)
    g = (0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3))
    for ez in range(nz - 1):
        for ey in range(ny - 1):
            for ex in range(nx - 1):
                for q in range(8):
                    s, t, w = g[q & 1], g[(q >> 1) & 1], g[q >> 2]
                    r = np.sqrt(((ex + s) * h[0]) ** 2 + ((ey + t) * h[1]) ** 2 + ((ez + w) * h[2]) ** 2)
                    sig = (3 * lam + 2 * mu) * m * 0.5 * (1 - np.tanh(l * (r - a)))
                    for c in range(8):
                        cx, cy, cz = c & 1, (c >> 1) & 1, c >> 2
                        Nx, Ny, Nz = (s if cx else 1 - s), (t if cy else 1 - t), (w if cz else 1 - w)
                        grad = ((1 if cx else -1) / h[0] * Ny * Nz, Nx * (1 if cy else -1) / h[1] * Nz,
                                Nx * Ny * (1 if cz else -1) / h[2])
                        for i in range(3):
                            ref[i, ez + cz, ey + cy, ex + cx] += h[0] * h[1] * h[2] / 8 * grad[i] * sig
    assert np.abs(f - ref).max() <= 1e-12 * np.abs(ref).max()


def test_uniform_eigenstrain_is_solved_exactly():
    # phi = 1 everywhere (a far beyond the domain): the free expansion u = m x
    # is stress free and meets the symmetry planes, so it is the solution
    shape, h = (6, 7, 5), (2.0, 1.5, 2.5)
    m = 0.01
    el = O.Elastic(shape, h)
    u, ok, _ = el.solve(E0, NU0, m, 1.0, 1e6, rtol=1e-14)
    assert ok
    x, y, z = coords(shape, h)
    ref = m * np.stack([x, y, z])
    assert np.abs(u - ref).max() <= 1e-11 * np.abs(ref).max()
    V, _, _ = el.sensitivity(E0, NU0, m, 1.0, 1e6, rtol=1e-14)
    V0 = 4 * h[0] * 6 * h[1] * 5 * h[2]
    assert V == pytest.approx(V0 * (1 + 3 * m), rel=1e-12)


def gauss_integral_of_phi(shape, h, l, a):
    nz, ny, nx = shape
    g = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    ex = (np.arange(nx - 1)[:, None] + g[None, :]).ravel() * h[0]
    ey = (np.arange(ny - 1)[:, None] + g[None, :]).ravel() * h[1]
    ez = (np.arange(nz - 1)[:, None] + g[None, :]).ravel() * h[2]
    Z, Y, X = np.meshgrid(ez, ey, ex, indexing="ij")
    r = np.sqrt(X * X + Y * Y + Z * Z)
    return float(np.sum(0.5 * (1 - np.tanh(l * (r - a))))) * h[0] * h[1] * h[2] / 8


def test_volume_equals_undeformed_plus_eigenstrain_integral():
    # a traction-free body (the symmetry planes make the octant one) has mean
    # stress zero, so with uniform moduli the mean strain is the mean
    # eigenstrain: V = V0 + 3 m int phi, for any E and nu; discretely the same
    # holds with the quadrature of phi, because x e_x, y e_y, z e_z are
    # admissible test fields
    shape, h = (9, 9, 9), (12.5, 12.5, 12.5)
    m, l, a = 0.01, 0.3, 40.0
    el = O.Elastic(shape, h)
    V0 = 8 * 12.5 * 8 * 12.5 * 8 * 12.5
    want = V0 + 3 * m * gauss_integral_of_phi(shape, h, l, a)
    for E, nu in ((E0, NU0), (3.0, 0.1), (50.0, 0.45)):
        V, grads, _ = el.sensitivity(E, nu, m, l, a, rtol=1e-13)
        assert V == pytest.approx(want, rel=1e-12, abs=1e-9 * (want - V0))
        assert abs(grads[0]) <= 1e-9 * (want - V0) and abs(grads[1]) <= 1e-9 * (want - V0)


def test_spherical_inclusion_radial_solution():
    # Eshelby / Timoshenko: a spherically symmetric dilatational eigenstrain
    # e*(r) in an unbounded isotropic body gives the radial displacement
    # u(r) = (1 + nu) / ((1 - nu) r^2) int_0^r e*(s) s^2 ds.  The octant of a
    # 100^3 cube with a = 12 is close to unbounded (the image term of a
    # traction-free outer boundary is ~ 2(1-2nu)/(1+nu) (a/b)^3 < 0.2 %); the
    # remaining difference is the O(h^2) discretisation error.
    n, L = 41, 100.0
    h = L / (n - 1)
    m, l, a = 0.01, 0.4, 12.0
    el = O.Elastic((n, n, n), h)
    u, ok, _ = el.solve(E0, NU0, m, l, a, rtol=1e-10)
    assert ok
    s = np.linspace(0, 60, 60001)
    phi = 0.5 * (1 - np.tanh(l * (s - a)))
    integ = np.concatenate([[0], np.cumsum(0.5 * (phi[1:] * s[1:] ** 2 + phi[:-1] * s[:-1] ** 2)
                                           * np.diff(s))])
    coef = (1 + NU0) / (1 - NU0) * m
    # nodes on the x axis up to r = 2a, where the outer boundary's image term
    # (relative size ~ 0.6 (r/b)^3 at r > a) stays below 1 %
    r = np.arange(1, 11) * h
    ref = coef * np.interp(r, s, integ) / r ** 2
    got = u[0, 0, 0, 1:11]
    assert np.allclose(got, ref, rtol=0.025)
    # inside the inclusion the strain is the uniform Eshelby value
    inner = got[: int(0.5 * a / h)] / r[: int(0.5 * a / h)]
    assert np.allclose(inner, coef / 3, rtol=0.005)
    # the same solution along the diagonal (radial symmetry of the discrete field)
    k = np.arange(1, 6)
    rd = np.sqrt(3) * k * h
    ud = np.sqrt(3) * u[0, k, k, k]  # |u| along (1,1,1) is sqrt(3) u_x there
    refd = coef * np.interp(rd, s, integ) / rd ** 2
    assert np.allclose(ud, refd, rtol=0.025)


def test_sensitivities_match_central_differences():
    shape, h = (7, 8, 9), (12.0, 11.0, 10.0)
    m, l, a = 0.01, 0.3, 35.0
    el = O.Elastic(shape, h)
    rng = np.random.default_rng(7)
    g = rng.standard_normal((3,) + shape)
    O0, grads, _ = el.sensitivity(E0, NU0, m, l, a, g=g, rtol=1e-14)
    # u does not depend on E (C and the load scale together)
    assert abs(grads[0]) <= 1e-10 * abs(O0) / E0
    for k, (E, nu) in enumerate(((E0, NU0),)):
        d = 1e-5
        Op, _, _ = el.sensitivity(E, nu + d, m, l, a, g=g, rtol=1e-14)
        Om, _, _ = el.sensitivity(E, nu - d, m, l, a, g=g, rtol=1e-14)
        assert grads[1] == pytest.approx((Op - Om) / (2 * d), rel=1e-6)
    # a point displacement: u_x at the far corner of the x axis
    gp = np.zeros((3,) + shape)
    gp[0, 0, 0, -1] = 1.0
    O1, g1, _ = el.sensitivity(E0, NU0, m, l, a, g=gp, rtol=1e-14)
    d = 1e-5
    Op, _, _ = el.sensitivity(E0, NU0 + d, m, l, a, g=gp, rtol=1e-14)
    Om, _, _ = el.sensitivity(E0, NU0 - d, m, l, a, g=gp, rtol=1e-14)
    assert g1[1] == pytest.approx((Op - Om) / (2 * d), rel=1e-6)
    assert abs(g1[1]) > 1e-3 * abs(O1)  # a genuinely nu-dependent objective
