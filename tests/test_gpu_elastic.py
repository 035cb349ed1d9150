"""GPU parity of the Eshelby-inclusion elasticity path (Eq. 3-4, Supp. 3 Eq.
III.1, objective Eq. 21-22) against the FP64 oracle: the stiffness operator
and the loads element by element on ragged grids, the CG solution, the
objective and its adjoint sensitivities; at the benchmark size the exact
uniform-eigenstrain solution and the volume identity."""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu

E0, NU0 = 22.5, 0.3


def rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def gpu(shape, h, **kw):
    import paper_2601_06079_gb300 as pf
    return pf.Elastic(shape, h, **kw)


def cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


@pytest.mark.parametrize("shape,h", [((5, 7, 9), (1.0, 1.3, 0.8)), ((17, 12, 33), (2.0, 2.0, 2.0)),
                                     ((2, 2, 2), (1.0, 1.0, 1.0)), ((40, 3, 2), (0.5, 1.5, 1.0))])
@pytest.mark.parametrize("constrain", [False, True])
def test_stiffness_apply_matches_oracle(shape, h, constrain):
    u = G.random_field(11, (3,) + shape)
    el = gpu(shape, h, E=E0, nu=NU0)
    got = el.apply(cu(u), constrain=constrain).cpu().numpy()
    lam, mu = O.Elastic.lame(E0, NU0)
    ref = O.Elastic(shape, h).apply(u.astype(np.float32).astype(np.float64), lam, mu)
    if constrain:
        ref[0, :, :, 0] = 0
        ref[1, :, 0, :] = 0
        ref[2, 0, :, :] = 0
    assert rel(got, ref) <= 2e-6


@pytest.mark.parametrize("shape,h,l,a", [((9, 10, 11), (10.0, 10.0, 10.0), 0.3, 40.0),
                                         ((6, 13, 7), (7.0, 4.0, 9.0), 1.0, 25.0)])
def test_loads_match_oracle(shape, h, l, a):
    m = 0.01
    el = gpu(shape, h, E=E0, nu=NU0, m=m, l=l, a=a)
    lam, mu = O.Elastic.lame(E0, NU0)
    oe = O.Elastic(shape, h)
    assert rel(el.load().cpu().numpy(), oe.rhs(lam, mu, m, l, a)) <= 2e-6
    V0, g = oe.volume_functional()
    assert rel(el.load(unit=True).cpu().numpy(), g) <= 2e-6


def test_solution_objective_and_sensitivities_match_oracle():
    shape, h = (17, 17, 17), (6.25, 6.25, 6.25)
    m, l, a = 0.01, 0.4, 30.0
    el = gpu(shape, h, E=E0, nu=NU0, m=m, l=l, a=a)
    oe = O.Elastic(shape, h)
    u_ref, ok, _ = oe.solve(E0, NU0, m, l, a, rtol=1e-12)
    assert ok
    u = el.solve(rtol=1e-6).cpu().numpy()
    assert el.stats.converged == 1
    assert rel(u, u_ref) <= 1e-5
    # a nu-dependent objective: u_x at the far end of the x axis, plus a random g
    for g in (np.eye(1, 3 * 17 ** 3, 16).reshape((3,) + shape),  # u_x at node (0, 0, 16)
              G.random_field(3, (3,) + shape)):
        O_ref, gr_ref, _ = oe.sensitivity(E0, NU0, m, l, a, g=g, rtol=1e-12)
        Og, gr, _ = el.sensitivity(g=cu(g), rtol=1e-6)
        assert Og == pytest.approx(O_ref, rel=1e-5)
        assert gr["nu"] == pytest.approx(gr_ref[1], rel=1e-4)
        # E-invariance of u: dO/dE is the solver residual over E
        assert abs(gr["E"]) <= 1e-5 * abs(O_ref) / E0
    # the volume: V and its (vanishing) sensitivities
    V_ref, _, _ = oe.sensitivity(E0, NU0, m, l, a, rtol=1e-12)
    V, gr, _ = el.sensitivity(rtol=1e-6)
    V0 = 16 ** 3 * 6.25 ** 3
    assert (V - V0) == pytest.approx(V_ref - V0, rel=1e-5)
    assert abs(gr["E"]) <= 1e-5 * (V_ref - V0) / E0
    assert abs(gr["nu"]) <= 1e-4 * (V_ref - V0)


@pytest.mark.parametrize("n", [129])
def test_full_size_exact_solutions(n):
    # the benchmark grid (129^3 nodes on the 100^3 cube): (1) phi = 1
    # everywhere: u = m x is the exact discrete solution; (2) the tanh
    # inclusion: V - V0 equals 3 m times the Gauss quadrature of phi (mean
    # strain of a traction-free body = mean eigenstrain); (3) sampled rows of
    # K u against the FP64 oracle's operator on a small crop around them
    h = 100.0 / (n - 1)
    m = 0.01
    el = gpu((n, n, n), h, E=E0, nu=NU0, m=m, l=1.0, a=1e6)
    u = el.solve(rtol=1e-6).cpu().numpy()
    z, y, x = np.meshgrid(*(np.arange(n) * h,) * 3, indexing="ij")
    ref = m * np.stack([x, y, z])
    assert np.abs(u - ref).max() <= 2e-5 * np.abs(ref).max()
    l, a = 0.5, 20.0
    el.set(l=l, a=a)
    V, gr, _ = el.sensitivity(rtol=1e-6)
    g = np.array([0.5 - 0.5 / np.sqrt(3), 0.5 + 0.5 / np.sqrt(3)])
    pts = ((np.arange(n - 1)[:, None] + g[None, :]).ravel() * h)
    r2 = pts[:, None, None] ** 2 + pts[None, :, None] ** 2 + pts[None, None, :] ** 2
    integ = float(np.sum(0.5 * (1 - np.tanh(l * (np.sqrt(r2) - a))))) * h ** 3 / 8
    V0 = 100.0 ** 3
    assert (V - V0) == pytest.approx(3 * m * integ, rel=2e-5)
    # K u rows: the operator is local, so rows of an interior crop (and of a
    # crop at the corner, where the boundary formula runs) equal the oracle's
    uf = G.random_field(5, (3, n, n, n))
    Ku = el.apply(cu(uf)).cpu().numpy()
    lam, mu = O.Elastic.lame(E0, NU0)
    for (z0, y0, x0) in ((60, 61, 62), (0, 0, 0), (n - 9, 0, n - 9)):
        crop = uf[:, z0:z0 + 9, y0:y0 + 9, x0:x0 + 9].astype(np.float32).astype(np.float64)
        r = O.Elastic((9, 9, 9), h).apply(crop, lam, mu)
        # rows whose 3x3x3 neighbourhood lies inside the crop, and whose
        # elements are all mesh elements (true at mesh faces the crop shares)
        zs = slice(1 if z0 else 0, 8 if z0 + 9 < n else 9)
        ys = slice(1 if y0 else 0, 8 if y0 + 9 < n else 9)
        xs = slice(1 if x0 else 0, 8 if x0 + 9 < n else 9)
        got = Ku[:, z0:z0 + 9, y0:y0 + 9, x0:x0 + 9][:, zs, ys, xs]
        assert rel(got, r[:, zs, ys, xs]) <= 2e-6


def test_invalid_arguments_are_rejected():
    from paper_2601_06079_gb300 import _lib
    import ctypes as C
    bad = [dict(n=(1, 5, 5)), dict(h=(0.0, 1.0, 1.0)), dict(E=0.0), dict(nu=0.5), dict(nu=-1.0),
           dict(m=float("nan"))]
    for b in bad:
        kw = dict(n=(5, 5, 5), h=(1.0, 1.0, 1.0), E=E0, nu=NU0, m=0.01, l=0.5, a=2.0)
        kw.update(b)
        e = _lib.pf_elastic((C.c_int64 * 3)(*kw["n"]), (C.c_double * 3)(*kw["h"]), kw["E"], kw["nu"],
                            kw["m"], kw["l"], kw["a"])
        st, _ = _lib.pf_elastic_workspace(e)
        assert st == _lib.PF_ERR_ARG


def test_solve_into_unaligned_buffer_matches_aligned():
    # the CG updates take a float4 path only when every vector is 16-byte
    # aligned; a displacement buffer offset by one float takes the scalar path
    shape, h = (9, 10, 11), (10.0, 10.0, 10.0)
    el = gpu(shape, h, E=E0, nu=NU0, m=0.01, l=0.3, a=40.0)
    u0 = el.solve(rtol=1e-6).clone()
    n = 3 * 9 * 10 * 11
    buf = torch.zeros(n + 1, device="cuda")
    u1 = buf[1:].view((3,) + shape)
    assert u1.data_ptr() % 16 != 0
    el.solve(u=u1, rtol=1e-6)
    assert rel(u1.cpu().numpy(), u0.cpu().numpy()) <= 1e-6


def test_zero_misfit_and_iteration_cap():
    # m = 0: the load vanishes, CG stops before its first iteration with u = 0,
    # V = V0 and zero sensitivities; a cap of 8 iterations on a real load
    # reports PF_ERR_NOT_CONVERGED with the stats of the partial solve
    import paper_2601_06079_gb300 as pf
    from paper_2601_06079_gb300 import _lib
    shape, h = (9, 9, 9), (12.5, 12.5, 12.5)
    el = gpu(shape, h, E=E0, nu=NU0, m=0.0, l=0.3, a=40.0)
    u = el.solve()
    assert el.stats.iterations == 0 and el.stats.converged == 1
    assert float(u.abs().max()) == 0.0
    V, gr, _ = el.sensitivity()
    assert V == pytest.approx(8 * 12.5 * 8 * 12.5 * 8 * 12.5, rel=1e-12)
    assert gr["E"] == 0.0 and gr["nu"] == 0.0
    el.set(m=0.01)
    with pytest.raises(pf.PFError) as ex:
        el.solve(rtol=1e-12, max_iter=8)
    assert ex.value.status == _lib.PF_ERR_NOT_CONVERGED
    assert el.stats.iterations == 8 and el.stats.converged == 0
    assert el.stats.final_residual < el.stats.initial_residual
