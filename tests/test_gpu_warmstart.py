"""The learned warm start: trained on the solver's own implicit trajectories
(other seeds), it must start Newton closer to the root than the plain U^n
guess on a held-out seed, need no more Newton iterations, and both starts
must converge to the same state within the Newton tolerance."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def test_warm_start_beats_plain_start_at_same_accuracy():
    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    from paper_2601_06079_gb300 import warmstart as WS

    n = 64
    solver = WS.grain_solver(n)
    data = WS.trajectories(solver, seeds=[101, 102, 103, 104, 105, 106], n_steps=14, n_grains=16)
    data = [t[2:].contiguous() for t in data]  # past the sharp-interface transient
    feats = [WS.inputs(solver, t) for t in data]
    surr = pf.Surrogate(features=True)
    surr.init(seed=7, last_layer_scale=0.0)
    losses = WS.train(surr, data, iters=800, crop=64, batch=4, lr=1e-3, seed=1, feats=feats)
    assert np.isfinite(losses).all()
    assert np.mean(losses[-20:]) < 0.5 * np.mean(losses[:20])

    U0 = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=16, n_op=8)).cuda()
    solver.step_implicit(U0, 2)
    Up, plain, r_plain = WS.run(solver, U0, 6, None, newton_rtol=1e-6)
    Uw, warm, r_warm = WS.run(solver, U0, 6, surr, newton_rtol=1e-6)
    assert np.mean(r_warm) < 0.6 * np.mean(r_plain), (np.mean(r_warm), np.mean(r_plain))
    assert warm["newton_iters"] <= plain["newton_iters"]
    diff = float(torch.linalg.norm(Uw - Up) / torch.linalg.norm(Up))
    assert diff <= 1e-5
