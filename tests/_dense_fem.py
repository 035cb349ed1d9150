"""Independent brute-force dense Q1 assembler (test-only, NumPy, FP64).

Written separately from the oracle to pin it: the quadrature points come from
numpy's Gauss-Legendre table (not from the closed form 1/sqrt 3), the shape
functions are written on physical coordinates, and everything is assembled
into dense matrices, so that a mistake in the oracle's reference-element
tables, its index arithmetic or its scatter shows up as a mismatch.
Only usable on tiny 2-D meshes (a few dozen nodes).
"""
import numpy as np


def _gauss01():
    x, w = np.polynomial.legendre.leggauss(2)
    return 0.5 * (x + 1.0), 0.5 * w


def _elements(nx, ny):
    for j in range(ny - 1):
        for i in range(nx - 1):
            yield i, j, [j * nx + i, j * nx + i + 1, (j + 1) * nx + i, (j + 1) * nx + i + 1]


def _shape(xl, yl, hx, hy):
    """Q1 values and physical gradients at local physical point (xl, yl)."""
    sx = [1 - xl / hx, xl / hx]
    sy = [1 - yl / hy, yl / hy]
    dsx = [-1 / hx, 1 / hx]
    dsy = [-1 / hy, 1 / hy]
    N, Gx, Gy = [], [], []
    for b in range(2):
        for a in range(2):
            N.append(sx[a] * sy[b])
            Gx.append(dsx[a] * sy[b])
            Gy.append(sx[a] * dsy[b])
    return np.array(N), np.array(Gx), np.array(Gy)


def _points(hx, hy):
    p, w = _gauss01()
    for qy in range(2):
        for qx in range(2):
            yield p[qx] * hx, p[qy] * hy, w[qx] * w[qy] * hx * hy


def assemble(nx, ny, hx, hy):
    """Dense consistent mass matrix and stiffness matrix."""
    n = nx * ny
    Mc = np.zeros((n, n))
    K = np.zeros((n, n))
    for _, _, nodes in _elements(nx, ny):
        for xl, yl, wt in _points(hx, hy):
            N, Gx, Gy = _shape(xl, yl, hx, hy)
            Mc[np.ix_(nodes, nodes)] += wt * np.outer(N, N)
            K[np.ix_(nodes, nodes)] += wt * (np.outer(Gx, Gx) + np.outer(Gy, Gy))
    return Mc, K


def nonlinear_vector(nx, ny, hx, hy, u, fprime):
    """F_i = integral of fprime(u_h) N_i by the 2x2 rule, assembled densely."""
    u = np.asarray(u, dtype=np.float64).ravel()
    F = np.zeros(nx * ny)
    for _, _, nodes in _elements(nx, ny):
        for xl, yl, wt in _points(hx, hy):
            N, _, _ = _shape(xl, yl, hx, hy)
            F[nodes] += wt * fprime(N @ u[nodes]) * N
    return F


def energy(nx, ny, hx, hy, u, f, kappa):
    u = np.asarray(u, dtype=np.float64).ravel()
    E = 0.0
    for _, _, nodes in _elements(nx, ny):
        for xl, yl, wt in _points(hx, hy):
            N, Gx, Gy = _shape(xl, yl, hx, hy)
            uq = N @ u[nodes]
            gx, gy = Gx @ u[nodes], Gy @ u[nodes]
            E += wt * (f(uq) + 0.5 * kappa * (gx * gx + gy * gy))
    return E


def mobility_stiffness(nx, ny, hx, hy, mfield, M=1.0):
    """Dense K_M with (K_M)_ij = sum_e sum_q w_q M(x_q) grad N_i . grad N_j, where
    the mobility at each Gauss point is the scalar M times the Q1 interpolant
    of the per-node field m (Eq. 9, mobility inside the divergence).  Both the
    points and the interpolation come from this module's own tables."""
    m = np.asarray(mfield, dtype=np.float64).ravel()
    n = nx * ny
    KM = np.zeros((n, n))
    for _, _, nodes in _elements(nx, ny):
        for xl, yl, wt in _points(hx, hy):
            N, Gx, Gy = _shape(xl, yl, hx, hy)
            Mq = M * float(N @ m[nodes])
            KM[np.ix_(nodes, nodes)] += wt * Mq * (np.outer(Gx, Gx) + np.outer(Gy, Gy))
    return KM
