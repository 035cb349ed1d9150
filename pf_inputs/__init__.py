"""Seeded synthetic inputs shared by the FP64 oracle, the tests and the bench.

This module holds only input generation: random fields, parameter samples and
initial conditions.  It contains none of the phase-field arithmetic (no
residual, no quadrature, no time step), so both sides of a parity check can
draw from it without sharing any of the method.

Every random number comes from SplitMix64 (Steele, Lea, Flood, "Fast
splittable pseudorandom number generators", OOPSLA 2014): state advances by
the golden-gamma constant and each output is the state passed through the
published 64-bit finaliser.  A stream is keyed by (seed, purpose) so that
different inputs of one workload never reuse numbers.  Doubles are drawn as
the top 53 bits times 2**-53, then rounded once to FP32 where the field is a
solver input, so the GPU and the oracle start from the same FP32 values (the
oracle widens them to FP64).

Shapes are (ny, nx) in 2-D and (nz, ny, nx) in 3-D, x fastest, matching the
node numbering n = (k*ny + j)*nx + i of the Q1 meshes.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

_PURPOSE = {
    "ac_init": 1,
    "ch_init": 2,
    "mobility": 3,
    "grains": 4,
    "batch": 5,
    "vector": 6,
    "target": 7,
    "surrogate": 8,
    "coupled": 9,
}


def _mix(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, count: int, purpose: str = "vector") -> np.ndarray:
    """`count` raw 64-bit outputs of the SplitMix64 stream keyed by (seed, purpose)."""
    key = (int(seed) * 0x100000001B3 + _PURPOSE[purpose] * 0x9E3779B1) & (2**64 - 1)
    with np.errstate(over="ignore"):
        state0 = _mix(np.array([key], dtype=np.uint64))[0]
        idx = np.arange(1, count + 1, dtype=np.uint64)
        return _mix(state0 + idx * _GAMMA)


def uniform(seed: int, count: int, lo: float = 0.0, hi: float = 1.0,
            purpose: str = "vector") -> np.ndarray:
    """FP64 uniform numbers in [lo, hi) from the keyed stream."""
    u = (splitmix64(seed, count, purpose) >> np.uint64(11)).astype(np.float64) * 2.0**-53
    return lo + (hi - lo) * u


def ac_initial(seed: int, shape, lo: float = 0.45, hi: float = 0.55) -> np.ndarray:
    """Allen-Cahn start field: phi0 ~ U[lo, hi) per node, rounded to FP32."""
    n = int(np.prod(shape))
    return uniform(seed, n, lo, hi, "ac_init").astype(np.float32).reshape(shape)


def ch_initial(seed: int, shape, mean: float = 0.5, amp: float = 0.05) -> np.ndarray:
    """Cahn-Hilliard start field: c0 = mean + U(-amp, amp) per node, rounded to FP32."""
    n = int(np.prod(shape))
    return (mean + uniform(seed, n, -amp, amp, "ch_init")).astype(np.float32).reshape(shape)


def random_field(seed: int, shape, lo: float = -1.0, hi: float = 1.0,
                 purpose: str = "vector") -> np.ndarray:
    """Generic FP32 test vector (directions for JVP / adjoint checks)."""
    n = int(np.prod(shape))
    return uniform(seed, n, lo, hi, purpose).astype(np.float32).reshape(shape)


def gaussian_mobility(seed: int, shape, h: float = 1.0, n_bumps: int = 8,
                      amp=(0.2, 0.8), width=(16.0, 64.0)) -> np.ndarray:
    """Smooth per-node mobility multiplier m(x) = 1 + sum_k a_k exp(-|x-x_k|^2 / (2 s_k^2)).

    a_k ~ U(amp), s_k ~ U(width) * h, centres uniform over the domain; FP32.
    """
    ny, nx = shape
    r = uniform(seed, 4 * n_bumps, 0.0, 1.0, "mobility").reshape(n_bumps, 4)
    Lx, Ly = (nx - 1) * h, (ny - 1) * h
    x = np.arange(nx) * h
    y = np.arange(ny) * h
    m = np.ones(shape, dtype=np.float64)
    for k in range(n_bumps):
        a = amp[0] + (amp[1] - amp[0]) * r[k, 0]
        s = (width[0] + (width[1] - width[0]) * r[k, 1]) * h
        cx, cy = r[k, 2] * Lx, r[k, 3] * Ly
        m += a * np.exp(-((x[None, :] - cx) ** 2 + (y[:, None] - cy) ** 2) / (2 * s * s))
    return m.astype(np.float32)


def voronoi_grains(seed: int, n: int = 128, n_seeds: int = 64, n_op: int = 8) -> np.ndarray:
    """3-D polycrystal start state for grain growth: (n_op, n, n, n) FP32.

    n_seeds Voronoi seeds uniform in the cube of n^3 nodes; every node belongs
    to its nearest seed's grain.  Grains are coloured with n_op order
    parameters by DSatur so that touching grains differ where the graph allows
    (the colour with the fewest conflicting neighbours otherwise).  eta_i = 1
    on nodes of grains coloured i and 0 elsewhere.
    """
    from scipy.spatial import cKDTree

    pts = uniform(seed, 3 * n_seeds, 0.0, n - 1.0, "grains").reshape(n_seeds, 3)
    g = np.arange(n, dtype=np.float64)
    zz, yy, xx = np.meshgrid(g, g, g, indexing="ij")
    _, lab = cKDTree(pts).query(np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1))
    lab = lab.reshape(n, n, n)
    adj = [set() for _ in range(n_seeds)]
    for ax in range(3):
        a = np.moveaxis(lab, ax, 0)
        p, q = a[:-1].ravel(), a[1:].ravel()
        d = p != q
        for u, v in set(zip(p[d].tolist(), q[d].tolist())):
            adj[u].add(v)
            adj[v].add(u)
    colour = [-1] * n_seeds
    for _ in range(n_seeds):
        best = max((i for i in range(n_seeds) if colour[i] < 0),
                   key=lambda i: (len({colour[j] for j in adj[i] if colour[j] >= 0}), len(adj[i]), -i))
        counts = [sum(1 for j in adj[best] if colour[j] == c) for c in range(n_op)]
        colour[best] = int(np.argmin(counts))
    col = np.asarray(colour)[lab]
    out = np.zeros((n_op, n, n, n), dtype=np.float32)
    for i in range(n_op):
        out[i][col == i] = 1.0
    return out


def batched_instances(seed: int, count: int = 256, sizes=(128, 256, 384, 512),
                      lo: float = 0.5, hi: float = 2.0):
    """Ensemble description: per instance (n, W, kappa, L).

    n uniform over `sizes` (square n x n node meshes); W, kappa, L
    log-uniform in [lo, hi].
    """
    r = uniform(seed, 4 * count, 0.0, 1.0, "batch").reshape(count, 4)
    ns = np.asarray(sizes)[np.minimum((r[:, 0] * len(sizes)).astype(int), len(sizes) - 1)]
    lw = np.log(lo) + (np.log(hi) - np.log(lo)) * r[:, 1:]
    par = np.exp(lw)
    return [dict(n=int(ns[i]), W=float(par[i, 0]), kappa=float(par[i, 1]), L=float(par[i, 2]))
            for i in range(count)]


def coupled_initial(seed: int, shape, n_disks: int = 12, c_mean: float = 0.6,
                    c_noise: float = 0.02, width: float = 2.0) -> np.ndarray:
    """Start state [c, eta] (2, ny, nx) FP32 for the coupled Allen-Cahn /
    Cahn-Hilliard model: eta = smooth disks (tanh profile of the given width in
    nodes, radii 5..15 % of the shorter side) in an eta = 0 matrix; c =
    c_mean + U(-c_noise, c_noise)."""
    ny, nx = shape
    r = uniform(seed, 3 * n_disks + ny * nx, 0.0, 1.0, "coupled")
    cx, cy = r[:n_disks] * (nx - 1), r[n_disks:2 * n_disks] * (ny - 1)
    rad = (0.05 + 0.10 * r[2 * n_disks:3 * n_disks]) * min(nx, ny)
    y, x = np.mgrid[0:ny, 0:nx].astype(np.float64)
    eta = np.zeros((ny, nx))
    for k in range(n_disks):
        d = np.sqrt((x - cx[k]) ** 2 + (y - cy[k]) ** 2)
        eta = np.maximum(eta, 0.5 * (1.0 - np.tanh((d - rad[k]) / width)))
    c = c_mean + c_noise * (2.0 * r[3 * n_disks:].reshape(ny, nx) - 1.0)
    return np.stack([c, eta]).astype(np.float32)
