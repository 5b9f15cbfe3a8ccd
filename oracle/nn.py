"""Oracle of the learned Poisson warm start (the growth direction that replaces the paper's
unspecified preconditioner, Sec. IV.C and App. G): a small convolutional network on a coarse
(eta, xi) grid, its squared-error loss, one Adam step, and the coarse/fine grid transfers.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain PyTorch CPU operations in float64;
the network is written out layer by layer.

Network: `depth` 3 x 3 convolutions, c_in -> width -> ... -> width -> 1 channel, bias, ReLU
after every layer but the last.  Padding: zero in eta (the first grid axis, radial: the wall
and the far field are not neighbours) and periodic in xi (the second axis, angular).
Parameters are one flat vector, layer by layer: weights (c_out, c_in, 3, 3) row-major, then
the bias (c_out).

Grid transfers between a fine (H 2^l) x (W 2^l) field and its coarse H x W image:
restriction averages each 2^l x 2^l block; prolongation applies l times the cell-centred
bilinear doubling: fine cell 2I takes 3/4 of coarse cell I and 1/4 of cell I - 1, fine cell
2I + 1 takes 3/4 of I and 1/4 of I + 1, along each axis, clamped at the ends of eta and
periodic in xi.
"""
from __future__ import annotations

import numpy as np
import torch

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def layer_shapes(c_in: int, width: int, depth: int):
    chans = [c_in] + [width] * (depth - 1) + [1]
    return [(chans[i + 1], chans[i]) for i in range(depth)]


def param_count(c_in: int, width: int, depth: int) -> int:
    return sum(co * ci * 9 + co for co, ci in layer_shapes(c_in, width, depth))


def unpack(params, c_in: int, width: int, depth: int):
    """[(w (co, ci, 3, 3), b (co))] views of the flat parameter tensor."""
    out, o = [], 0
    for co, ci in layer_shapes(c_in, width, depth):
        w = params[o:o + co * ci * 9].reshape(co, ci, 3, 3)
        o += co * ci * 9
        b = params[o:o + co]
        o += co
        out.append((w, b))
    return out


def conv3x3(x, w, b):
    """y[n, co, i, j] = b[co] + sum_{ci, a, c} w[co, ci, a, c] x[n, ci, i + a - 1, j + c - 1], with
    x = 0 outside 0 <= i < H and j taken modulo W."""
    xp = torch.cat([x[..., -1:], x, x[..., :1]], dim=3)            # periodic in xi
    xp = torch.nn.functional.pad(xp, (0, 0, 1, 1))                 # zero in eta
    return torch.nn.functional.conv2d(xp, w) + b.view(1, -1, 1, 1)


def forward(params, x, c_in: int, width: int, depth: int):
    h = x
    layers = unpack(params, c_in, width, depth)
    for k, (w, b) in enumerate(layers):
        h = conv3x3(h, w, b)
        if k < depth - 1:
            h = torch.relu(h)
    return h


def loss_and_grad(params, x, y, c_in: int, width: int, depth: int):
    """Mean squared error over every output entry and its gradient in the parameters."""
    p = params.detach().clone().requires_grad_(True)
    pred = forward(p, x, c_in, width, depth)
    loss = torch.mean((pred - y) ** 2)
    loss.backward()
    return float(loss.detach()), p.grad.detach().clone()


def adam_step(params, grad, m, v, t: int, lr: float):
    """One Adam update (Kingma & Ba 2015) with step count t >= 1; returns new (params, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * grad
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * grad * grad
    mh = m / (1.0 - ADAM_B1 ** t)
    vh = v / (1.0 - ADAM_B2 ** t)
    return params - lr * mh / (torch.sqrt(vh) + ADAM_EPS), m, v


def restrict(fine: np.ndarray, levels: int) -> np.ndarray:
    f = np.asarray(fine, dtype=np.float64)
    s = 2 ** levels
    H, W = f.shape[0] // s, f.shape[1] // s
    return f.reshape(H, s, W, s).mean(axis=(1, 3))


def _double(c: np.ndarray) -> np.ndarray:
    H, W = c.shape
    f = np.empty((2 * H, 2 * W))
    t = np.empty((2 * H, W))
    for I in range(H):
        t[2 * I] = 0.75 * c[I] + 0.25 * c[max(I - 1, 0)]
        t[2 * I + 1] = 0.75 * c[I] + 0.25 * c[min(I + 1, H - 1)]
    for J in range(W):
        f[:, 2 * J] = 0.75 * t[:, J] + 0.25 * t[:, (J - 1) % W]
        f[:, 2 * J + 1] = 0.75 * t[:, J] + 0.25 * t[:, (J + 1) % W]
    return f


def prolong(coarse: np.ndarray, levels: int) -> np.ndarray:
    f = np.asarray(coarse, dtype=np.float64)
    for _ in range(levels):
        f = _double(f)
    return f
