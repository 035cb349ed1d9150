"""GPU parity at the size limits of the 2-D explicit path (Eq. 11-12).

- A mesh just under the 2^31 - 1 node cap of `pf_create_mesh` (32,771 x
  65,521 nodes): the ghost-padded working planes exceed 2^31 elements, so
  every offset has to be 64-bit.  The start field repeats a seeded tile, which
  gives closed forms for the whole-mesh energy and mass (sums of oracle
  energies of a few periodic sub-meshes), and the oracle reproduces sampled
  nodes after k steps from windows of radius 2k + margin.
- Meshes at the per-axis limit (2^20 nodes) with the minimum width (2 nodes
  for AC, 3 for CH) in either orientation, checked element by element.
"""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu

REL_L2 = 1e-5


def _pf():
    import paper_2601_06079_gb300 as pf
    return pf


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


PAR = {"ac": dict(W=1.0, kappa=1.0, mobility=1.0, dt=0.01),
       "ch": dict(W=1.0, kappa=0.5, mobility=1.0, dt=1e-3)}


def _oracle(model, shape):
    p = PAR[model]
    return O.Problem(shape, W=p["W"], kappa=p["kappa"], mob=p["mobility"])


def _oracle_steps(model, u0, k):
    P = _oracle(model, u0.shape)
    dt = PAR[model]["dt"]
    return P.ch_explicit(u0, dt, k) if model == "ch" else P.ac_explicit(u0, dt, k)


# ------------------------------------------------------------ node-count cap

NY, NX = 32_771, 65_521      # 2,147,220,691 nodes <= 2^31 - 1
PY, PX = 1_031, 1_033        # period of the tiled start field


def _tile(model):
    return (G.ch_initial(21, (PY, PX)) if model == "ch"
            else G.ac_initial(21, (PY, PX))).astype(np.float32)


def _periodic(T, ys, xs):
    return T[np.ix_(np.asarray(ys) % PY, np.asarray(xs) % PX)]


def _energy_closed_form(model, T, ny=NY, nx=NX):
    # E_h is a sum over elements (Eq. 5-6 with 2x2 Gauss); the element with
    # lower corner (y, x) sees the tile's values at (y mod PY, x mod PX), so
    # with n - 1 = q P + r elements per axis the sum splits into q^2 full
    # periods, strips and one corner block, each the energy of a periodic
    # sub-mesh of (rows + 1) x (cols + 1) nodes.
    qy, ry = divmod(ny - 1, PY)
    qx, rx = divmod(nx - 1, PX)

    def E(ra, rb):
        if ra == 0 or rb == 0:
            return 0.0
        sub = _periodic(T, range(ra + 1), range(rb + 1)).astype(np.float64)
        return _oracle(model, sub.shape).energy(sub)

    return qy * qx * E(PY, PX) + qy * E(PY, rx) + qx * E(ry, PX) + E(ry, rx)


def _mass_closed_form(T, ny=NY, nx=NX):
    # lumped mass m_i = h^2 w_x w_y with w = 1/2 at the end nodes (h = 1)
    def weights(n, p):
        w = np.ones(n)
        w[0] = w[-1] = 0.5
        return np.bincount(np.arange(n) % p, weights=w, minlength=p)
    return float(weights(ny, PY) @ T.astype(np.float64) @ weights(nx, PX))


@pytest.mark.parametrize("model", ["ch", "ac"])
def test_mesh_at_the_node_cap(model):
    free, _ = torch.cuda.mem_get_info()
    if free < 40 * 2**30:
        pytest.skip("needs about 30 GB of free device memory")
    pf = _pf()
    T = _tile(model)
    Tt = torch.from_numpy(T).cuda()
    strip = Tt.repeat(1, -(-NX // PX))[:, :NX]
    u = torch.empty((NY, NX), dtype=torch.float32, device="cuda")
    for y0 in range(0, NY, PY):
        r = min(PY, NY - y0)
        u[y0:y0 + r] = strip[:r]
    del strip, Tt
    s = pf.Solver((NY, NX), h=1.0, model=model)
    s.set_params(**PAR[model])

    E0, M0 = s.energy(u)
    assert abs(E0 - _energy_closed_form(model, T)) <= 1e-6 * abs(E0)
    assert abs(M0 - _mass_closed_form(T)) <= 1e-10 * abs(M0)

    k = 3
    s.step_explicit(u, k)
    E1, M1 = s.energy(u)
    assert E1 < E0  # gradient flow with a stable step
    if model == "ch":
        assert abs(M1 - M0) <= 1e-7 * abs(M0)

    # sampled nodes: after k steps a node depends on start data within 2k
    # nodes; windows touching the mesh edge keep the true zero-flux boundary,
    # the last rows lie past 2^31 elements of the working planes
    R = 2 * k + 4
    centres = [(0, 0), (0, NX - 1), (NY - 1, 0), (NY - 1, NX - 1), (0, NX // 2),
               (NY - 1, NX // 3), (NY // 2, 0), (NY // 3, NX - 1), (NY // 2, NX // 2),
               (NY - 10, 40_000), (PY * 7, PX * 11), (PY * 7 - 1, PX * 11 - 1)]
    for cy, cx in centres:
        y0, y1 = max(0, cy - R), min(NY, cy + R + 1)
        x0, x1 = max(0, cx - R), min(NX, cx + R + 1)
        win = _periodic(T, range(y0, y1), range(x0, x1))
        ref = _oracle_steps(model, win, k)
        sy = slice(0 if y0 == 0 else 2 * k + 1, win.shape[0] if y1 == NY else win.shape[0] - 2 * k - 1)
        sx = slice(0 if x0 == 0 else 2 * k + 1, win.shape[1] if x1 == NX else win.shape[1] - 2 * k - 1)
        g = u[y0:y1, x0:x1].cpu().numpy()[sy, sx]
        r = ref[sy, sx]
        assert g.size > 0
        assert rel_l2(g, r) <= REL_L2, (cy, cx)
    s.close()
    del u, s
    torch.cuda.empty_cache()


# ------------------------------------------------------- per-axis node limit

@pytest.mark.parametrize("model,shape", [("ch", (3, 1 << 20)), ("ch", (1 << 20, 3)),
                                         ("ac", (2, 1 << 20)), ("ac", (1 << 20, 2))])
def test_thinnest_meshes_at_the_axis_limit(model, shape):
    u0 = (G.ch_initial(22, shape) if model == "ch" else G.ac_initial(22, shape, 0.2, 0.8))
    k = 12
    pf = _pf()
    s = pf.Solver(shape, h=1.0, model=model)
    s.set_params(**PAR[model])
    t = torch.from_numpy(u0).cuda()
    s.step_explicit(t, k)
    out = t.cpu().numpy()
    ref = _oracle_steps(model, u0, k)
    assert rel_l2(out, ref) <= REL_L2
    if model == "ch":
        assert np.abs(out - ref).max() <= 2e-6


# Rows of blocks beyond the 65,535 that grid.y holds: 2^20 node rows in the
# two-pass form (8-row blocks) and in the mobility-field step and its adjoint
# (16-row tiles); wide rows of 2^20 nodes for contrast.

def _cu(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("shape", [(1 << 20, 3), (3, 1 << 20)])
def test_two_pass_form_at_the_axis_limit(shape):
    c0 = G.ch_initial(23, shape)
    k = 6
    pf = _pf()
    s = pf.Solver(shape, h=1.0, model="ch")
    s.set_params(**PAR["ch"])
    s.set_form("two_pass")
    t = _cu(c0)
    s.step_explicit(t, k)
    assert rel_l2(t.cpu().numpy(), _oracle_steps("ch", c0, k)) <= REL_L2


def test_mobility_field_step_and_adjoint_on_the_tallest_mesh():
    shape = (1 << 20, 3)
    mob = G.gaussian_mobility(24, shape, h=1.0)
    c0, target = G.ch_initial(25, shape), G.ch_initial(26, shape)
    pf = _pf()
    s = pf.Solver(shape, model="ch")
    s.set_params(W=1.1, kappa=0.6, mobility=0.9, dt=0.02, mobility_field=_cu(mob))
    P = O.Problem(shape, W=1.1, kappa=0.6, mob=0.9, mob_field=mob)
    k = 4
    t = _cu(c0)
    s.step_explicit(t, k)
    assert rel_l2(t.cpu().numpy(), P.ch_explicit(c0, 0.02, k)) <= REL_L2
    loss, g = s.adjoint(_cu(c0), _cu(target), k, 2, want_state=True)
    oloss, og = P.ch_adjoint(c0, target, 0.02, k)
    assert abs(loss - oloss) <= 1e-5 * abs(oloss)
    for key in ("kappa", "W", "M"):
        assert abs(g[key] - og[key]) <= 1e-4 * abs(og[key]), key
    assert rel_l2(g["mobility_field"].cpu().numpy(), og["mob_field"]) <= 1e-4
    assert rel_l2(g["c0"].cpu().numpy(), og["c0"]) <= 1e-4


def test_ensemble_of_more_instances_than_grid_rows():
    # 65,600 instances (more than grid.y holds) of 4 x 4 and 5 x 7 nodes with
    # per-instance W, kappa, L; sampled instances against the oracle, the
    # persistent and per-step forms bitwise equal
    count = 65_600
    shapes = [(4, 4) if i % 2 == 0 else (5, 7) for i in range(count)]
    par = [dict(W=0.5 + (i % 7) / 7, kappa=0.5 + (i % 5) / 5, L=0.5 + (i % 3) / 3, dt=0.01)
           for i in range(count)]
    flat = G.ac_initial(27, (count * 51,))
    fields, o = [], 0
    for sh in shapes:
        n = sh[0] * sh[1]
        fields.append(flat[o:o + n].reshape(sh))
        o += n
    pf = _pf()
    e = pf.Ensemble(shapes)
    e.set_params(par)
    st0 = e.pack(fields)
    k = 20
    a = e.step(st0.clone(), k, "persistent")
    b = e.step(st0.clone(), k, "per_step")
    assert torch.equal(a, b)
    out = e.unpack(a)
    for i in [0, 1, 65_533, 65_534, 65_535, 65_536, 65_537, count - 2, count - 1, 40_001]:
        p = par[i]
        ref = O.Problem(shapes[i], W=p["W"], kappa=p["kappa"], mob=p["L"]).ac_explicit(
            fields[i], 0.01, k)
        assert rel_l2(out[i].cpu().numpy(), ref) <= REL_L2, i
    e.close()


# ------------------------------------------- 3-D vectors past 2^31 values

FC = dict(alpha=1.0, beta=1.0, gamma=1.5)


def _tiled3(T, n, P3):
    """(c, n, n, n) device array repeating the (c,) + P3 tile T."""
    t = torch.from_numpy(T).cuda()
    big = t.repeat(1, *[-(-n // p) for p in P3])
    out = big[:, :n, :n, :n].contiguous()
    del big
    return out


def _window3(T, P3, zs, ys, xs):
    return T[:, np.asarray(zs) % P3[0]][:, :, np.asarray(ys) % P3[1]][:, :, :, np.asarray(xs) % P3[2]]


def _check_windows(n, centres, gpu_and_oracle):
    """Compare sampled 5^3-node windows; gpu_and_oracle(rng) -> pairs of
    (device array, oracle window array); faces that are not mesh faces drop."""
    for cz, cy, cx in centres:
        lo = [max(0, c - 2) for c in (cz, cy, cx)]
        hi = [min(n, c + 3) for c in (cz, cy, cx)]
        rng = [range(a, b) for a, b in zip(lo, hi)]
        keep = (slice(None),) + tuple(slice(0 if a == 0 else 1, (b - a) if b == n else (b - a) - 1)
                                      for a, b in zip(lo, hi))
        sl = (slice(None),) + tuple(slice(a, b) for a, b in zip(lo, hi))
        for gpu, ref in gpu_and_oracle(rng):
            g = gpu[sl].cpu().numpy()[keep]
            r = ref[keep]
            assert g.size > 0
            assert rel_l2(g, r) <= 2e-6, (cz, cy, cx)


def test_fan_chen_jvp_and_residual_past_2_31_values():
    # 648^3 nodes x 8 order parameters: one vector holds 2.18e9 values, so the
    # field offsets exceed 2^31.  U, U^n and v repeat seeded tiles; J v and R
    # at a node involve only the 8 elements around it, so the oracle
    # reproduces sampled nodes from 5^3-node windows (window faces that are
    # not mesh faces are left out).
    free, _ = torch.cuda.mem_get_info()
    if free < 80 * 2**30:
        pytest.skip("needs about 60 GB of free device memory")
    n, nf, P3 = 648, 8, (37, 41, 43)
    TU = G.random_field(31, (nf,) + P3, 0.0, 1.0)
    TN = G.random_field(32, (nf,) + P3, 0.0, 1.0)
    TV = G.random_field(33, (nf,) + P3)

    pf = _pf()
    s = pf.Solver((n, n, n), h=1.0, model="fanchen", n_fields=nf)
    s.set_params(W=1.0, kappa=0.9, mobility=1.1, dt=0.5, shift=0.0, **FC)
    U, v = _tiled3(TU, n, P3), _tiled3(TV, n, P3)
    Jv = s.jvp(U, v)
    del v
    torch.cuda.empty_cache()
    Un = _tiled3(TN, n, P3)
    R = s.implicit_residual(Un, U)
    centres = [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n // 2), (n // 2, n // 2, n // 2),
               (n - 2, n - 1, 1), (300, 0, n - 1), (n - 1, 500, 37 * 5)]

    def pairs(rng):
        Uw, Nw, Vw = (_window3(T, P3, *rng) for T in (TU, TN, TV))
        P = O.Problem(Uw.shape[1:], h=1.0, energy="fan_chen", nf=nf, kappa=0.9, mob=1.1,
                      W=1.0, **FC)
        return ((Jv, P.implicit_jvp(0.5, Uw, Vw)), (R, P.implicit_residual(0.5, Nw, Uw)))

    _check_windows(n, centres, pairs)
    s.close()
    del U, Un, Jv, R, s
    torch.cuda.empty_cache()


# The remaining operators on meshes at the axis limit (1-D tile grids): the
# coupled step (Eq. 7) in both orientations, the 2-D implicit operators and the
# 3-D Fan-Chen J v with 2^20 nodes along z and an odd field count.

@pytest.mark.parametrize("shape", [(1 << 20, 3), (3, 1 << 20)])
def test_coupled_step_at_the_axis_limit(shape):
    U0 = G.coupled_initial(41, shape)
    par = dict(kappa=0.3, mobility=1.0, mobility2=150.0, dt=1e-3)
    pf = _pf()
    s = pf.Solver(shape, h=1.0, model="coupled")
    s.set_params(**par)
    t = _cu(U0)
    s.step_explicit(t, 6)
    P = O.Problem(shape, energy="coupled", kappa=0.3, mob=1.0, mob2=150.0)
    ref = P.coupled_explicit(U0, 1e-3, 6)
    got = t.cpu().numpy()
    for f in range(2):
        assert rel_l2(got[f], ref[f]) <= REL_L2, f


def test_implicit_operators_at_the_axis_limit():
    pf = _pf()
    shape = (1 << 20, 3)
    s = pf.Solver(shape, h=1.0, model="ac")
    s.set_params(W=1.0, kappa=0.9, mobility=1.1, dt=0.5)
    P = O.Problem(shape, W=1.0, kappa=0.9, mob=1.1)
    U, Un = G.ac_initial(42, shape, 0.2, 0.8), G.ac_initial(43, shape, 0.2, 0.8)
    v = G.random_field(44, shape)
    assert rel_l2(s.jvp(_cu(U), _cu(v)).cpu().numpy(), P.implicit_jvp(0.5, U, v)) <= 2e-6
    assert rel_l2(s.implicit_residual(_cu(Un), _cu(U)).cpu().numpy(),
                  P.implicit_residual(0.5, Un, U)) <= 2e-6
    shape3, nf = (1 << 20, 2, 3), 3
    s3 = pf.Solver(shape3, h=1.0, model="fanchen", n_fields=nf)
    s3.set_params(W=1.0, kappa=0.9, mobility=1.1, dt=0.5, shift=0.0, **FC)
    P3 = O.Problem(shape3, h=1.0, energy="fan_chen", nf=nf, kappa=0.9, mob=1.1, W=1.0, **FC)
    U3 = G.random_field(45, (nf,) + shape3, 0.0, 1.0)
    v3 = G.random_field(46, (nf,) + shape3)
    assert rel_l2(s3.jvp(_cu(U3), _cu(v3)).cpu().numpy(), P3.implicit_jvp(0.5, U3, v3)) <= 2e-6


def test_elastic_stiffness_past_2_31_values():
    # 896^3 nodes x 3 displacement components: 2.16e9 values per vector.  K u
    # at a node involves only its 8 elements, so 5^3-node windows of a tiled
    # random u are reproduced by the oracle (no constraints).
    free, _ = torch.cuda.mem_get_info()
    if free < 50 * 2**30:
        pytest.skip("needs about 30 GB of free device memory")
    n, P3 = 896, (37, 41, 43)
    E, nu = 22.5, 0.3
    T = G.random_field(51, (3,) + P3)
    pf = _pf()
    el = pf.Elastic((n, n, n), 1.0, E=E, nu=nu)
    u = _tiled3(T, n, P3)
    Ku = el.apply(u)
    lam, mu = O.Elastic.lame(E, nu)

    def pairs(rng):
        uw = _window3(T, P3, *rng).astype(np.float64)
        return ((Ku, O.Elastic(uw.shape[1:], 1.0).apply(uw, lam, mu)),)

    _check_windows(n, [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, n // 2), (n // 2, n // 2, n // 2),
                       (n - 2, n - 1, 1), (700, 0, n - 1), (n - 1, 600, 37 * 7)], pairs)
    del u, Ku, el
    torch.cuda.empty_cache()
