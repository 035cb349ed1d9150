"""GPU parity of the fused coupled Allen-Cahn / Cahn-Hilliard step (Eq. 7 with
the Supp. 3 polynomials, explicit Euler with the lumped mass) against the
FP64 oracle: ragged small meshes element by element, a 1024^2 mesh over
whole fields, conservation of c, and the error paths."""
import numpy as np
import pytest
import torch

import oracle as O
import pf_inputs as G

pytestmark = pytest.mark.gpu

PAR = dict(kappa=0.3, mobility=1.0, mobility2=150.0, dt=1e-3)


def rel(a, b):
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / np.linalg.norm(b))


def run(U0, h, n_steps):
    import paper_2601_06079_gb300 as pf
    s = pf.Solver(U0.shape[1:], h=h, model="coupled")
    s.set_params(**PAR)
    t = torch.from_numpy(np.ascontiguousarray(U0, np.float32)).cuda()
    s.step_explicit(t, n_steps)
    torch.cuda.synchronize()
    return t.cpu().numpy(), s, t


def oracle(U0, h, n_steps):
    P = O.Problem(U0.shape[1:], h=h, energy="coupled", kappa=PAR["kappa"], mob=PAR["mobility"],
                  mob2=PAR["mobility2"])
    return P.coupled_explicit(U0, PAR["dt"], n_steps), P


@pytest.mark.parametrize("shape,h", [((33, 41), 1.0), ((67, 35), (0.9, 1.2)), ((3, 4), 1.0),
                                     ((100, 130), 1.0), ((3, 9), 1.0), ((6, 3), 1.0),
                                     ((17, 33), 1.0)])
def test_coupled_matches_oracle(shape, h):
    U0 = G.coupled_initial(5, shape)
    got, _, _ = run(U0, h, 150)
    ref, _ = oracle(U0, h, 150)
    for f in range(2):
        assert rel(got[f], ref[f]) <= 1e-5, (f, rel(got[f], ref[f]))


def test_coupled_1024_whole_fields():
    U0 = G.coupled_initial(7, (1024, 1024))
    got, _, _ = run(U0, 1.0, 40)
    ref, _ = oracle(U0, 1.0, 40)
    for f in range(2):
        assert rel(got[f], ref[f]) <= 1e-5
    assert np.abs(got[1] - U0[1]).max() > 1e-3  # the interfaces moved


def test_coupled_conserves_c():
    U0 = G.coupled_initial(9, (256, 256))
    got, _, _ = run(U0, 1.0, 2000)
    P = O.Problem((256, 256), energy="coupled", kappa=0.3, mob=1.0, mob2=150.0)
    m0, m1 = P.mass_integral(U0[0].astype(np.float64)), P.mass_integral(got[0])
    assert abs(m1 - m0) <= 1e-6 * abs(m0)
    # the discrete energy went down
    assert P.energy(got) < P.energy(U0.astype(np.float64))


def test_coupled_errors():
    import paper_2601_06079_gb300 as pf
    from paper_2601_06079_gb300 import _lib
    s = pf.Solver((16, 16), model="coupled")
    with pytest.raises(pf.PFError):
        s.set_params(kappa=0.3, mobility=1.0, dt=1e-3)  # no M_eta
    s.set_params(**PAR)
    t = torch.zeros(2 * 16 * 16, device="cuda")
    with pytest.raises(pf.PFError):
        s.energy(t)
    st, ctx, ws = _lib.pf_create_mesh(2, [16, 16], [1.0, 1.0], _lib.PF_MODEL_COUPLED, 1, 0)
    assert st == _lib.PF_ERR_ARG
