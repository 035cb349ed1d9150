"""Independent reference of the surrogate U-Net in plain PyTorch autograd
(test-only): the same layer sequence, weight layout and loss, evaluated in
FP64 on the CPU, to check the library's whole-network gradient."""
import torch
import torch.nn.functional as F

LAYERS = [(16, 32, 1, 0), (32, 32, 1, 0), (32, 32, 1, 1), (32, 32, 1, 1), (32, 32, 1, 2),
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


def forward(params, x):
    """x: [B][8][D][H][W] -> 16-channel increment estimate."""
    Ws = unpack(params)
    h = torch.cat([x, torch.zeros_like(x)], dim=1)

    def conv(l, t):
        w, b = Ws[l]
        y = F.conv3d(t, w, b, padding=1)
        return torch.relu(y) if LAYERS[l][2] else y

    up = lambda t: t.repeat_interleave(2, 2).repeat_interleave(2, 3).repeat_interleave(2, 4)
    a = conv(1, conv(0, h)); s0 = a
    a = conv(3, conv(2, F.avg_pool3d(a, 2))); s1 = a
    a = conv(5, conv(4, F.avg_pool3d(a, 2))); s2 = a
    a = conv(7, conv(6, F.avg_pool3d(a, 2)))
    a = conv(9, conv(8, up(a) + s2))
    a = conv(11, conv(10, up(a) + s1))
    a = conv(13, conv(12, up(a) + s0))
    return conv(14, a)


def loss(params, x, y):
    out = forward(params, x)[:, :8]
    return ((out - (y - x)) ** 2).mean()
