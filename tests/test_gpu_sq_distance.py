"""pf_sq_distance, the library's sum of squared differences (the learned warm
start's output unit without history): against an FP64 NumPy sum of the same
FP32 differences, bitwise repeatable, over sizes from one value to several
grid-stride passes with ragged tails."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _ref(a, b):
    d = (a - b).astype(np.float64)  # the difference in FP32, as the kernel forms it
    return float(np.sum(d * d))


@pytest.mark.parametrize("n", [1, 255, 257, 262_144, 1_000_003, 9_437_185])
def test_matches_fp64_sum(n):
    import paper_2601_06079_gb300 as pf
    import pf_inputs as G
    a = G.uniform(11, n, -1.0, 1.0, "vector").astype(np.float32)
    b = (a + G.uniform(12, n, -1e-3, 1e-3, "vector")).astype(np.float32)
    ta, tb = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    v = pf.sq_distance(ta, tb)
    ref = _ref(a, b)
    assert abs(v - ref) <= 1e-9 * ref, (v, ref)
    assert pf.sq_distance(ta, tb) == v  # fixed summation order
    assert pf.sq_distance(ta, ta) == 0.0


def test_increment_scale_of_a_trajectory():
    import pf_inputs as G
    from paper_2601_06079_gb300 import warmstart as WS
    t = [torch.from_numpy(G.uniform(s, 5 * 8 * 16 ** 3, 0.0, 1.0, "vector")
                          .astype(np.float32).reshape(5, 8, 16, 16, 16)).cuda()
         for s in (1, 2)]
    s, n = 0.0, 0
    for x in t:
        h = x.cpu().numpy()
        s += _ref(h[1:], h[:-1])
        n += h[1:].size
    ref = (s / n) ** 0.5
    assert abs(WS.increment_scale(t) - ref) <= 1e-10 * ref


def test_empty_and_bad_arguments():
    import paper_2601_06079_gb300 as pf
    e = torch.empty(0, device="cuda")
    assert pf.sq_distance(e, e) == 0.0
    with pytest.raises(ValueError):
        pf.sq_distance(torch.zeros(4, device="cuda"), torch.zeros(5, device="cuda"))
    with pytest.raises(ValueError):
        pf.sq_distance(torch.zeros(4, device="cuda", dtype=torch.float64),
                       torch.zeros(4, device="cuda", dtype=torch.float64))
