"""CPU pins of the references that the size-limit GPU tests build: the
closed-form energy and mass of a mesh that repeats a tile, and the oracle
windows that stand in for whole-mesh oracle results.  Each is compared with
the oracle run on the whole (small) tiled mesh."""
import numpy as np
import pytest

import oracle as O
import pf_inputs as G
from tests import test_gpu_extreme_sizes as X


@pytest.mark.parametrize("model", ["ch", "ac"])
@pytest.mark.parametrize("ny,nx", [(2500, 3100), (1032, 1034), (1031, 2067), (3, 5), (1031, 1040)])
def test_tiled_energy_and_mass_closed_forms(model, ny, nx):
    # sums over whole periods, strips and a corner block of the tile equal the
    # oracle's element sum and lumped-mass sum over the tiled mesh
    T = X._tile(model)
    u = X._periodic(T, range(ny), range(nx)).astype(np.float64)
    P = X._oracle(model, u.shape)
    E, M = P.energy(u), P.mass_integral(u)
    assert abs(X._energy_closed_form(model, T, ny, nx) - E) <= 1e-12 * abs(E)
    assert abs(X._mass_closed_form(T, ny, nx) - M) <= 1e-13 * abs(M)


class _Host:
    """Stands in for a device array in the window helper (slicing, .cpu().numpy())."""

    def __init__(self, a):
        self.a = a

    def __getitem__(self, k):
        return _Host(self.a[k])

    def cpu(self):
        return self

    def numpy(self):
        return self.a


def test_windows_reproduce_whole_mesh_operators(monkeypatch):
    # J v, R (Fan-Chen, 8 fields) and K u (elasticity) on 5^3-node windows of
    # a tiled mesh equal the whole-mesh oracle at the nodes the helper keeps
    n, P3, nf = 11, (3, 4, 5), 8
    TU = G.random_field(31, (nf,) + P3, 0.0, 1.0)
    TN = G.random_field(32, (nf,) + P3, 0.0, 1.0)
    TV = G.random_field(33, (nf,) + P3)
    TE = G.random_field(51, (3,) + P3)
    full = [X._window3(T, P3, range(n), range(n), range(n)).astype(np.float64)
            for T in (TU, TN, TV, TE)]
    P = O.Problem((n, n, n), h=1.0, energy="fan_chen", nf=nf, kappa=0.9, mob=1.1, W=1.0, **X.FC)
    lam, mu = O.Elastic.lame(22.5, 0.3)
    whole = {"jv": P.implicit_jvp(0.5, full[0], full[2]),
             "r": P.implicit_residual(0.5, full[1], full[0]),
             "ku": O.Elastic((n, n, n), 1.0).apply(full[3], lam, mu)}
    worst = []
    monkeypatch.setattr(X, "rel_l2", lambda a, b: worst.append(
        float(np.abs(a - b).max() / np.abs(b).max())) or worst[-1])

    def pairs(rng):
        Uw, Nw, Vw, Ew = (X._window3(T, P3, *rng) for T in (TU, TN, TV, TE))
        Pw = O.Problem(Uw.shape[1:], h=1.0, energy="fan_chen", nf=nf, kappa=0.9, mob=1.1,
                       W=1.0, **X.FC)
        return ((_Host(whole["jv"]), Pw.implicit_jvp(0.5, Uw, Vw)),
                (_Host(whole["r"]), Pw.implicit_residual(0.5, Nw, Uw)),
                (_Host(whole["ku"]), O.Elastic(Ew.shape[1:], 1.0).apply(Ew.astype(np.float64),
                                                                        lam, mu)))

    X._check_windows(n, [(0, 0, 0), (n - 1, n - 1, n - 1), (n - 1, 0, 5), (5, 5, 5),
                         (n - 2, n - 1, 1), (3, 0, n - 1)], pairs)
    assert len(worst) == 18 and max(worst) <= 1e-13
