"""Pins of the learned-warm-start oracle (oracle/nn.py) against brute force and closed forms."""
import numpy as np
import pytest
import torch

from oracle import nn as N
from paper_2507_05222_gb300 import inputs


def brute_conv(x, w, b):
    """The convolution written as plain loops: zero outside the eta range, xi periodic."""
    n_, ci_, H, W = x.shape
    co_ = w.shape[0]
    y = np.zeros((n_, co_, H, W))
    for n in range(n_):
        for co in range(co_):
            for i in range(H):
                for j in range(W):
                    s = b[co]
                    for ci in range(ci_):
                        for a in range(3):
                            ii = i + a - 1
                            if not 0 <= ii < H:
                                continue
                            for c in range(3):
                                s += w[co, ci, a, c] * x[n, ci, ii, (j + c - 1) % W]
                    y[n, co, i, j] = s
    return y


def test_conv_equals_brute_force():
    g = inputs.rng(1)
    x = g.standard_normal((2, 3, 5, 6))
    w = g.standard_normal((4, 3, 3, 3))
    b = g.standard_normal(4)
    y = N.conv3x3(torch.tensor(x), torch.tensor(w), torch.tensor(b)).numpy()
    assert np.allclose(y, brute_conv(x, w, b), rtol=1e-13, atol=1e-13)


def test_conv_is_periodic_in_xi_only():
    g = inputs.rng(2)
    x = torch.tensor(g.standard_normal((1, 2, 6, 8)))
    w, b = torch.tensor(g.standard_normal((3, 2, 3, 3))), torch.tensor(g.standard_normal(3))
    y = N.conv3x3(x, w, b)
    # a circular shift in xi commutes with the layer
    assert torch.allclose(N.conv3x3(torch.roll(x, 3, dims=3), w, b), torch.roll(y, 3, dims=3), atol=1e-13)
    # a shift in eta does not (the wall and the far field are not neighbours)
    assert not torch.allclose(N.conv3x3(torch.roll(x, 1, dims=2), w, b), torch.roll(y, 1, dims=2), atol=1e-6)


def test_forward_layers_and_parameter_layout():
    c_in, width, depth = 3, 5, 4
    n = N.param_count(c_in, width, depth)
    assert n == (5 * 3 * 9 + 5) + 2 * (5 * 5 * 9 + 5) + (1 * 5 * 9 + 1)
    g = inputs.rng(3)
    p = torch.tensor(g.standard_normal(n) * 0.3)
    x = torch.tensor(g.standard_normal((2, c_in, 4, 6)))
    h = x.numpy()
    for k, (w, b) in enumerate(N.unpack(p, c_in, width, depth)):
        h = brute_conv(h, w.numpy(), b.numpy())
        if k < depth - 1:
            h = np.maximum(h, 0.0)
    assert np.allclose(N.forward(p, x, c_in, width, depth).numpy(), h, rtol=1e-12, atol=1e-12)


def test_gradient_against_finite_differences():
    c_in, width, depth = 2, 3, 3
    g = inputs.rng(4)
    p = torch.tensor(g.standard_normal(N.param_count(c_in, width, depth)) * 0.5)
    x = torch.tensor(g.standard_normal((2, c_in, 4, 5)))
    y = torch.tensor(g.standard_normal((2, 1, 4, 5)))
    loss, grad = N.loss_and_grad(p, x, y, c_in, width, depth)
    h = 1e-6
    for i in list(range(0, len(p), 7)):
        e = torch.zeros_like(p)
        e[i] = h
        lp = float(torch.mean((N.forward(p + e, x, c_in, width, depth) - y) ** 2))
        lm = float(torch.mean((N.forward(p - e, x, c_in, width, depth) - y) ** 2))
        assert abs((lp - lm) / (2 * h) - float(grad[i])) <= 1e-6 * max(1.0, abs(float(grad[i])))
    assert loss == pytest.approx(float(torch.mean((N.forward(p, x, c_in, width, depth) - y) ** 2)))


def test_adam_first_step_closed_form():
    # after one step from m = v = 0 the bias-corrected moments are g and g^2: the step is
    # lr g / (|g| + eps)
    g = torch.tensor([3.0, -2.0, 1e-3, 0.0])
    p = torch.tensor([1.0, 1.0, 1.0, 1.0])
    p1, m, v = N.adam_step(p, g, torch.zeros(4), torch.zeros(4), 1, 0.01)
    expect = p - 0.01 * g / (g.abs() + N.ADAM_EPS)
    assert torch.allclose(p1, expect, rtol=1e-15, atol=1e-15)
    assert torch.allclose(m, 0.1 * g) and torch.allclose(v, 0.001 * g * g)


def test_restrict_prolong():
    g = inputs.rng(5)
    f = g.standard_normal((16, 32))
    c = N.restrict(f, 2)
    assert c.shape == (4, 8)
    assert np.isclose(c[1, 3], f[4:8, 12:16].mean())
    # prolongation keeps constants and reproduces a function linear in eta away from the two
    # eta ends, and any function of xi with zero second differences (constants) exactly
    assert np.allclose(N.prolong(np.full((4, 8), 2.5), 3), 2.5)
    H, W = 8, 8
    lin = np.add.outer(np.arange(H, dtype=float), np.zeros(W))
    fine = N.prolong(lin, 1)
    # fine cell i sits at coarse position i / 2 - 1/4
    expect = np.add.outer(np.arange(2 * H) / 2.0 - 0.25, np.zeros(2 * W))
    assert np.allclose(fine[1:-1], expect[1:-1])
    # periodic in xi: a field periodic in xi stays periodic (shift commutes)
    c2 = g.standard_normal((4, 8))
    assert np.allclose(N.prolong(np.roll(c2, 1, axis=1), 2), np.roll(N.prolong(c2, 2), 4, axis=1))
    # restriction after prolongation of one level preserves the mean of every coarse cell's
    # neighbourhood weights: the total is preserved
    assert np.isclose(N.prolong(c2, 1).sum() / 4.0, c2.sum())
