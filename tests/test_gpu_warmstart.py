"""The learned warm start (history-2 surrogate: a learned correction to
quadratic extrapolation through the last three states), trained on the
solver's own implicit trajectories from other seeds, against the plain U^n
start on a held-out seed: Newton must start closer to the root, need fewer
Newton iterations, and every start must converge to the same state within
the Newton tolerance."""
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
    data = WS.trajectories(solver, seeds=[101, 102, 103, 104, 105, 106], n_steps=30, n_grains=16)
    surr = pf.Surrogate(history=2)
    surr.init(seed=7, last_layer_scale=0.0)
    losses = WS.train(surr, data, iters=600, crop=64, batch=4, lr=1e-4, seed=1, stiff=0.5)
    assert np.isfinite(losses).all()

    U0 = torch.from_numpy(G.voronoi_grains(1, n=n, n_seeds=16, n_op=8)).cuda()
    Up, plain, r_plain = WS.run(solver, U0, 40, None, newton_rtol=1e-6)
    Uw, warm, r_warm = WS.run(solver, U0, 40, surr, newton_rtol=1e-6)
    # from the third step on the surrogate has its full history
    assert np.median(r_warm[2:]) < 0.5 * np.median(r_plain[2:]), (r_warm[:6], r_plain[:6])
    assert warm["newton_iters"] < 0.75 * plain["newton_iters"], (warm, plain)
    diff = float(torch.linalg.norm(Uw - Up) / torch.linalg.norm(Up))
    assert diff <= 1e-5
