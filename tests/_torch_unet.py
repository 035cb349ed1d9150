"""Independent reference of the surrogate U-Net in plain PyTorch autograd
(test-only): the same layer sequence, weight layout and loss, evaluated in
FP64 on the CPU, to check the library's whole-network gradient."""
import torch
import torch.nn.functional as F

LAYERS = [(32, 32, 1, 0), (32, 32, 1, 0), (32, 32, 1, 1), (32, 32, 1, 1), (32, 32, 1, 2),
          (32, 32, 1, 2), (32, 32, 1, 3), (32, 32, 1, 3), (32, 32, 1, 2), (32, 32, 1, 2),
          (32, 32, 1, 1), (32, 32, 1, 1), (32, 32, 1, 0), (32, 32, 1, 0), (32, 16, 0, 0)]


def unpack(params):
    out, o = [], 0
    for ci, co, _, _ in LAYERS:
        w = params[o:o + 27 * co * ci].reshape(3, 3, 3, co, ci).permute(3, 4, 0, 1, 2)
        o += 27 * co * ci
        b = params[o:o + co]
        o += co
        out.append((w, b))
    return out


class _Bf16Store(torch.autograd.Function):
    """A buffer the library keeps in BF16: the value is rounded on the way
    forward, and the gradient the library stores for it is rounded on the way
    back (both round to nearest even)."""

    @staticmethod
    def forward(ctx, t):
        return t.to(torch.bfloat16).to(t.dtype)

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


class _Bf16Grad(torch.autograd.Function):
    """An FP32 value whose gradient the library stores in BF16 (the network
    output: the loss gradient is rounded before the backward pass)."""

    @staticmethod
    def forward(ctx, t):
        return t.clone()

    @staticmethod
    def backward(ctx, g):
        return g.to(torch.bfloat16).to(g.dtype)


def bf16_weights(params):
    """The parameters as the library's kernels use them: the convolution
    weights rounded to BF16 (round to nearest even), the biases FP32."""
    out, o = params.clone(), 0
    for ci, co, _, _ in LAYERS:
        n = 27 * co * ci
        out[o:o + n] = params[o:o + n].to(torch.bfloat16).to(params.dtype)
        o += n + co
    return out


def forward(params, x, bf16=False):
    """x: [B][8 or 16][D][H][W] network input -> 16-channel output.  With bf16,
    every buffer the library stores in BF16 (activations, pooled and upsampled
    sums, and their gradients) is rounded as it is there; the weights and the
    input are expected already rounded by the caller."""
    Ws = unpack(params)
    pad = torch.zeros((x.shape[0], 32 - x.shape[1]) + tuple(x.shape[2:]), dtype=x.dtype)
    h = torch.cat([x, pad], dim=1)
    q = _Bf16Store.apply if bf16 else (lambda t: t)
    if bf16:
        h = q(h)

    def conv(l, t):
        w, b = Ws[l]
        y = F.conv3d(t, w, b, padding=1)
        y = torch.relu(y) if LAYERS[l][2] else y
        return q(y) if l < len(LAYERS) - 1 else (_Bf16Grad.apply(y) if bf16 else y)

    up = lambda t: t.repeat_interleave(2, 2).repeat_interleave(2, 3).repeat_interleave(2, 4)
    pool = lambda t: q(F.avg_pool3d(t, 2))
    a = conv(1, conv(0, h)); s0 = a
    a = conv(3, conv(2, pool(a))); s1 = a
    a = conv(5, conv(4, pool(a))); s2 = a
    a = conv(7, conv(6, pool(a)))
    a = conv(9, conv(8, q(up(a) + s2)))
    a = conv(11, conv(10, q(up(a) + s1)))
    a = conv(13, conv(12, q(up(a) + s0)))
    return conv(14, a)


def loss(params, x, y, bf16=False, x_target=None):
    """Mean squared error of the increment net(x) against y - x; the library
    forms the target from the unrounded state, passed as x_target."""
    out = forward(params, x, bf16)[:, :8]
    xt = x if x_target is None else x_target
    return ((out - (y - xt)) ** 2).mean()


def history_input(x):
    """[U^n; U^{n-1}; ...] -> (network input [U^n, dU_1 / s, dU_2 / s, ...], s per
    sample), dU_k = U^{n-k+1} - U^{n-k}, s = RMS of dU_1 over the sample."""
    h = x.shape[1] // 8 - 1
    st = [x[:, 8 * k:8 * (k + 1)] for k in range(h + 1)]
    du = [st[k] - st[k + 1] for k in range(h)]
    s = du[0].pow(2).mean(dim=(1, 2, 3, 4), keepdim=True).sqrt()
    return torch.cat([st[0]] + [d / s for d in du], dim=1), s


def output_scale(x, s):
    """Output unit of the correction: s on top of linear extrapolation; on top of
    quadratic extrapolation the RMS of the second difference U^n - 2 U^{n-1} +
    U^{n-2} over the sample, floored at 1e-3 s."""
    h = x.shape[1] // 8 - 1
    if h < 2:
        return s
    st = [x[:, 8 * k:8 * (k + 1)] for k in range(3)]
    r = (st[0] - 2 * st[1] + st[2]).pow(2).mean(dim=(1, 2, 3, 4), keepdim=True).sqrt()
    return torch.maximum(r, 1e-3 * s)


def extrapolate(x):
    """Linear (2 states) or quadratic (3 states) extrapolation to the next state."""
    h = x.shape[1] // 8 - 1
    st = [x[:, 8 * k:8 * (k + 1)] for k in range(h + 1)]
    return 2 * st[0] - st[1] if h == 1 else 3 * st[0] - 3 * st[1] + st[2]


def stiff_apply(e, c):
    """(I + c K) e for fields e [B][F][D][H][W] on the unit-spaced mesh: K is the
    assembled Q1 stiffness with natural boundaries, written as the 27-point
    stencil on the mirror-extended field times the lumped-mass weight
    (1/2 per boundary axis)."""
    B, F_, D, H, W = e.shape
    k = torch.zeros(3, 3, 3, dtype=e.dtype)
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                n = (dz != 1) + (dy != 1) + (dx != 1)
                k[dz, dy, dx] = {0: 8.0 / 3.0, 1: 0.0, 2: -1.0 / 6.0, 3: -1.0 / 12.0}[n]
    t = F.pad(e.reshape(B * F_, 1, D, H, W), (1, 1, 1, 1, 1, 1), mode="reflect")
    se = F.conv3d(t, k[None, None]).reshape(B, F_, D, H, W)
    w = torch.ones(D, H, W, dtype=e.dtype)
    w[0] *= 0.5
    w[-1] *= 0.5
    w[:, 0] *= 0.5
    w[:, -1] *= 0.5
    w[:, :, 0] *= 0.5
    w[:, :, -1] *= 0.5
    return e + c * w * se


def loss_history(params, h, x, y, s, stiff=0.0, bf16=False):
    """Loss in units of s of the guess extrapolate(x) + s * net(h) against y,
    the error weighted by (I + stiff K)."""
    out = forward(params, h, bf16)[:, :8]
    return (stiff_apply(out - (y - extrapolate(x)) / s, stiff) ** 2).mean()
