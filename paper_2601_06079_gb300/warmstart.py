"""Learned warm start for the implicit grain-growth step (Eq. 13-14).

The solver generates its own training data: implicit trajectories of the
Fan-Chen grain-growth model from seeded Voronoi starts.  A surrogate with
history h (pf_surrogate_*) sees the current state and h earlier ones and
predicts a correction to polynomial extrapolation through them (h = 2:
U^{n+1} ~ 3 U^n - 3 U^{n-1} + U^{n-2} + c * net), in units c of the RMS of
the second difference: where the trajectory is nearly quadratic the
correction shrinks with it, and slow late stages of coarsening weigh as much
in training as the fast early ones.  Its output is the first Newton iterate.
While fewer earlier states exist the surrogate runs with what there is (the
second step of a run uses one earlier state), and the plain start U^n is the
fallback on the first step and without a surrogate.  Newton's converged residual is the measure: every start
is iterated to the same tolerance, so the gain shows up as fewer Newton /
GMRES iterations and less wall time at the same accuracy.

All arithmetic runs in the library's kernels; this module only orchestrates
calls, copies states into the network's input buffer and draws crop positions
from the seeded generator.
"""
from __future__ import annotations

import time

import numpy as np
import torch

import pf_inputs as G

from . import Solver, Surrogate, sq_distance

FANCHEN = dict(kappa=1.0, mobility=1.0, alpha=1.0, beta=1.0, gamma=1.5, shift=0.0)


def grain_solver(n, dt=0.5, device="cuda"):
    s = Solver((n, n, n), model="fanchen", n_fields=8, device=device)
    s.set_params(dt=dt, **FANCHEN)
    return s


def trajectories(solver, seeds, n_steps, n_grains=64):
    """Implicit trajectories from Voronoi starts; returns a list of [steps+1, 8, n, n, n]
    CUDA tensors (float32)."""
    n = solver.shape[0]
    out = []
    for sd in seeds:
        U = torch.from_numpy(G.voronoi_grains(sd, n=n, n_seeds=n_grains, n_op=8)).cuda()
        traj = [U.clone()]
        for _ in range(n_steps):
            solver.step_implicit(U, 1)
            traj.append(U.clone())
        out.append(torch.stack(traj))
    return out


def increment_scale(trajs):
    """RMS of U^{n+1} - U^n over the training pairs (output unit without history);
    the squared increments are summed by the library (pf_sq_distance)."""
    s, n = 0.0, 0
    for t in trajs:
        s += sq_distance(t[1:], t[:-1])
        n += t[1:].numel()
    return (s / n) ** 0.5


def train(surr, trajs, iters, crop=64, batch=4, lr=1e-3, seed=0, log_every=0, lr_final=None,
          stiff=0.0):
    """Adam on random (state, crop) samples; crops are crop^3 (the volume itself
    when it is not larger).  The learning rate decays geometrically to
    lr_final (default lr / 10).  stiff > 0 weighs the error by (I + stiff K),
    the linear part of the implicit Jacobian relative to its mass term
    (stiff = dt L kappa / h^2)."""
    rng = np.random.default_rng(seed)
    hist = surr.history
    surr.out_scale = 1.0 if hist else increment_scale(trajs)
    assert all(t.shape[0] >= hist + 2 for t in trajs), "trajectories too short for the history"
    lr_final = lr / 10 if lr_final is None else lr_final
    losses = []
    for it in range(iters):
        xs, ys = [], []
        for _ in range(batch):
            t = trajs[rng.integers(len(trajs))]
            k = rng.integers(hist, t.shape[0] - 1)
            n = t.shape[-1]
            c = min(crop, n)
            o = [rng.integers(n - c + 1) for _ in range(3)]
            sl = (slice(None), slice(o[0], o[0] + c), slice(o[1], o[1] + c), slice(o[2], o[2] + c))
            xs.append(torch.cat([t[k - j][sl] for j in range(hist + 1)]))
            ys.append(t[k + 1][sl])
        x = torch.stack(xs).contiguous()
        y = torch.stack(ys).contiguous()
        rate = lr * (lr_final / lr) ** (it / max(1, iters - 1))
        losses.append(surr.train_step(x, y, lr=rate, stiff=stiff))
        if log_every and (it + 1) % log_every == 0:
            print(f"  train {it + 1}: loss {losses[-1]:.3e}", flush=True)
    return losses


def run(solver, U0, n_steps, surr=None, newton_rtol=1e-5):
    """n_steps implicit steps from U0 with the plain start (surr None) or the
    learned one; returns (final state, totals, per-step initial residuals).
    A history surrogate falls back to the plain start on the first step and
    uses the earlier states there are until it has all of them."""
    U = U0.clone()
    tot = dict(newton_iters=0, gmres_iters=0, seconds=0.0, predict_seconds=0.0)
    r0 = []
    guess = torch.empty_like(U)
    h = surr.history if surr is not None else 0
    x = None
    if surr is not None:
        x = torch.empty((1, 8 * (h + 1)) + tuple(U.shape[1:]), device=U.device)
    avail = 0  # earlier states held in x[0, 8:]
    for _ in range(n_steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        g = None
        if surr is not None and (avail > 0 or h == 0):
            x[0, :8].copy_(U)
            surr.predict(x[:, :8 * (avail + 1)], out=guess[None])
            torch.cuda.synchronize()
            tot["predict_seconds"] += time.perf_counter() - t0
            g = guess
        if h > 0:  # U^n becomes the first earlier state of the next step
            for j in range(min(avail, h - 1), 0, -1):
                x[0, 8 * (j + 1):8 * (j + 2)].copy_(x[0, 8 * j:8 * (j + 1)])
            x[0, 8:16].copy_(U)
            avail = min(avail + 1, h)
        st = solver.step_implicit(U, 1, guess=g, newton_rtol=newton_rtol)
        torch.cuda.synchronize()
        tot["seconds"] += time.perf_counter() - t0
        tot["newton_iters"] += st["newton_iters"]
        tot["gmres_iters"] += st["gmres_iters"]
        r0.append(st["initial_residual"])
    return U, tot, r0
