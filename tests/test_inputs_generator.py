"""CPU pins of the seeded input generator shared by the oracle and the GPU
tests: the SplitMix64 finaliser against the published outputs of the stream
started at state 0, the keyed streams' independence and reproducibility, and
the ranges of the derived fields."""
import numpy as np

import pf_inputs as G


def test_splitmix64_matches_published_outputs_from_state_zero():
    # SplitMix64 from state 0 yields 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    # 0x06C45D188009454F (the stream advances by the golden gamma, then mixes)
    with np.errstate(over="ignore"):
        z = G._mix(np.arange(1, 4, dtype=np.uint64) * G._GAMMA)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_keyed_streams_are_reproducible_prefix_stable_and_distinct():
    a = G.splitmix64(7, 1000, "vector")
    assert np.array_equal(a, G.splitmix64(7, 1000, "vector"))
    assert np.array_equal(a[:10], G.splitmix64(7, 10, "vector"))  # prefix of a longer draw
    for other in (G.splitmix64(8, 1000, "vector"), G.splitmix64(7, 1000, "ac_init")):
        assert np.count_nonzero(a == other) == 0


def test_uniform_fields_stay_in_range_with_the_right_mean():
    u = G.uniform(3, 200_000, -2.0, 5.0)
    assert u.min() >= -2.0 and u.max() < 5.0
    assert abs(u.mean() - 1.5) < 0.03
    c = G.ch_initial(1, (64, 80))
    assert c.dtype == np.float32 and c.shape == (64, 80)
    assert c.min() >= 0.45 - 1e-7 and c.max() <= 0.55 + 1e-7  # FP32 rounding of the bounds
    f = G.ac_initial(2, (33, 17), 0.2, 0.8)
    assert f.min() >= 0.2 - 1e-7 and f.max() <= 0.8 + 1e-7
