"""Pins of the oracle's 3x3x3 convolution (surrogate layers) without a GPU:
an independent NumPy brute force (shifted slices of a zero-padded array), the
delta kernel (identity / shift), linearity, the adjoint dot-product identity
<conv(x), y> = <x, conv^T(y)>, and central differences of a scalar loss for
the weight gradient."""
import numpy as np

import oracle as O
import pf_inputs as G


def brute(x, w, b):
    ci, d, h, ww = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (1, 1)))
    y = np.zeros((w.shape[0], d, h, ww)) + b[:, None, None, None]
    for kz in range(3):
        for ky in range(3):
            for kx in range(3):
                sl = xp[:, kz:kz + d, ky:ky + h, kx:kx + ww]
                y += np.einsum("oi,izyx->ozyx", w[:, :, kz, ky, kx], sl)
    return y


def rnd(seed, shape):
    return G.random_field(seed, shape).astype(np.float64)


def test_conv_matches_numpy_brute_force():
    x, w, b = rnd(1, (3, 5, 6, 7)), rnd(2, (4, 3, 3, 3, 3)), rnd(3, (4,))
    np.testing.assert_allclose(O.conv3d(x, w, b), brute(x, w, b), rtol=1e-12, atol=1e-12)


def test_delta_kernel_is_a_shift():
    x = rnd(4, (2, 4, 5, 6))
    w = np.zeros((2, 2, 3, 3, 3))
    w[0, 0, 1, 1, 1] = 1.0      # identity on channel 0
    w[1, 1, 1, 1, 2] = 1.0      # channel 1 shifted: y(x) = x(x + 1)
    y = O.conv3d(x, w)
    np.testing.assert_array_equal(y[0], x[0])
    np.testing.assert_array_equal(y[1][..., :-1], x[1][..., 1:])
    assert np.all(y[1][..., -1] == 0)


def test_adjoint_identity_and_linearity():
    x, dy, w = rnd(5, (3, 4, 5, 6)), rnd(6, (2, 4, 5, 6)), rnd(7, (2, 3, 3, 3, 3))
    lhs = np.vdot(O.conv3d(x, w), dy)
    rhs = np.vdot(x, O.conv3d_bwd_data(dy, w))
    assert abs(lhs - rhs) < 1e-11 * abs(lhs)
    x2 = rnd(8, x.shape)
    np.testing.assert_allclose(O.conv3d(2 * x + x2, w), 2 * O.conv3d(x, w) + O.conv3d(x2, w),
                               rtol=1e-12, atol=1e-12)


def test_weight_gradient_matches_central_fd():
    x, w, b, t = rnd(9, (2, 3, 4, 5)), rnd(10, (3, 2, 3, 3, 3)), rnd(11, (3,)), rnd(12, (3, 3, 4, 5))
    loss = lambda w_, b_: 0.5 * np.sum((O.conv3d(x, w_, b_) - t) ** 2)
    dy = O.conv3d(x, w, b) - t
    dw, db = O.conv3d_bwd_weight(x, dy)
    eps = 1e-6
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 1, 1), (1, 0, 2, 0, 1), (0, 1, 1, 2, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        fd = (loss(wp, b) - loss(wm, b)) / (2 * eps)
        assert abs(dw[idx] - fd) < 1e-6 * max(1.0, abs(fd))
    for o in range(3):
        bp, bm = b.copy(), b.copy()
        bp[o] += eps
        bm[o] -= eps
        assert abs(db[o] - (loss(w, bp) - loss(w, bm)) / (2 * eps)) < 1e-6 * max(1, abs(db[o]))


def test_torch_reference_stiffness_weight_is_the_assembled_q1_stiffness():
    # the loss weighting (I + c K) of the surrogate's torch reference, against
    # the oracle's element-by-element assembly of K (natural boundaries, h = 1)
    import torch
    from tests import _torch_unet as R
    rng = np.random.default_rng(3)
    e = rng.standard_normal((1, 2, 5, 6, 7))
    got = R.stiff_apply(torch.from_numpy(e), 1.0).numpy() - e
    P = O.Problem((5, 6, 7), h=1.0, energy="double_well", nf=1, mob=1.0)
    for f in range(2):
        ref = P.mobility_stiffness_apply(e[0, f])
        assert np.abs(got[0, f] - ref).max() <= 1e-12 * np.abs(ref).max()
