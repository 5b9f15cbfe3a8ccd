"""The learned warm start's network and grid transfers through the C ABI against the oracle
(oracle/nn.py, float64): forward pass, loss and gradient, the Adam update, input/output
scaling, training progress, restriction and prolongation, moments."""
import numpy as np
import pytest
import torch

from oracle import nn as N
from paper_2507_05222_gb300 import inputs

pytestmark = pytest.mark.gpu
C_IN, WIDTH, DEPTH = 3, 32, 4


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2507_05222_gb300 import qtt
    return qtt.Context(0)


def he_params(seed, c_in=C_IN, width=WIDTH, depth=DEPTH):
    """He-scaled normal weights, zero biases (drawn on the host, passed in)."""
    g = inputs.rng(seed)
    out = []
    for co, ci in N.layer_shapes(c_in, width, depth):
        out.append(g.standard_normal(co * ci * 9) * np.sqrt(2.0 / (ci * 9)))
        out.append(np.zeros(co))
    return np.concatenate(out).astype(np.float32)


def rel(a, b):
    a = np.asarray(a, dtype=np.float64).ravel(); b = np.asarray(b, dtype=np.float64).ravel()
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_forward_matches_oracle(ctx):
    from paper_2507_05222_gb300 import qtt
    p = he_params(1)
    p[-1] = 0.3                                  # a non-zero output bias
    net = qtt.NN(ctx, C_IN, WIDTH, DEPTH, p)
    x = inputs.rng(2).standard_normal((2, C_IN, 16, 32)).astype(np.float32)
    y = net.predict(x)
    ref = N.forward(torch.tensor(p, dtype=torch.float64), torch.tensor(x, dtype=torch.float64), C_IN, WIDTH, DEPTH)
    assert rel(y, ref.numpy()) < 1e-5
    assert np.array_equal(net.params(), p)


def test_scaling_matches_oracle(ctx):
    from paper_2507_05222_gb300 import qtt
    p = he_params(3)
    net = qtt.NN(ctx, C_IN, WIDTH, DEPTH, p)
    shift, scale, out = np.array([1.0, -0.5, 2.0]), np.array([4.0, 0.25, 10.0]), 0.01
    net.set_scaling(shift, scale, out)
    x = inputs.rng(4).standard_normal((1, C_IN, 8, 16)).astype(np.float32)
    xs = (x.astype(np.float64) - shift[None, :, None, None]) * scale[None, :, None, None]
    ref = out * N.forward(torch.tensor(p, dtype=torch.float64), torch.tensor(xs), C_IN, WIDTH, DEPTH).numpy()
    assert rel(net.predict(x), ref) < 1e-5


def test_loss_gradient_and_adam_match_oracle(ctx):
    from paper_2507_05222_gb300 import qtt
    p = he_params(5)
    net = qtt.NN(ctx, C_IN, WIDTH, DEPTH, p)
    g = inputs.rng(6)
    x = g.standard_normal((2, C_IN, 16, 16)).astype(np.float32)
    y = g.standard_normal((2, 1, 16, 16)).astype(np.float32)
    pt = torch.tensor(p, dtype=torch.float64)
    loss_ref, grad_ref = N.loss_and_grad(pt, torch.tensor(x, dtype=torch.float64),
                                         torch.tensor(y, dtype=torch.float64), C_IN, WIDTH, DEPTH)
    lr = 1e-3
    loss = net.train_step(x, y, lr)
    grad = net.grad()
    assert abs(loss - loss_ref) <= 1e-5 * loss_ref
    assert rel(grad, grad_ref.numpy()) < 1e-4
    # the device's Adam update equals the oracle's formula applied to the device's gradient
    # (one step from zero moments: sign-sensitive where |g| is tiny, hence the same gradient)
    p1, _, _ = N.adam_step(pt, torch.tensor(grad, dtype=torch.float64), torch.zeros_like(pt), torch.zeros_like(pt),
                           1, lr)
    assert np.abs(net.params().astype(np.float64) - p1.numpy()).max() <= 1e-6 * lr + 1e-7


def test_training_reduces_the_loss(ctx):
    """A student with the teacher's architecture learns a fixed random teacher network's map."""
    from paper_2507_05222_gb300 import qtt
    teacher = he_params(7, width=8, depth=3)
    net = qtt.NN(ctx, C_IN, 8, 3, he_params(8, width=8, depth=3))
    g = inputs.rng(9)
    xs = g.standard_normal((16, C_IN, 16, 16)).astype(np.float32)
    ys = N.forward(torch.tensor(teacher, dtype=torch.float64), torch.tensor(xs, dtype=torch.float64), C_IN, 8,
                   3).numpy().astype(np.float32)
    losses = [net.train_step(xs[(4 * k) % 16:(4 * k) % 16 + 4], ys[(4 * k) % 16:(4 * k) % 16 + 4], 3e-3)
              for k in range(400)]
    assert np.mean(losses[-20:]) < 0.3 * np.mean(losses[:20])


def test_grid_transfers_match_oracle(ctx):
    from paper_2507_05222_gb300 import qtt
    g = inputs.rng(10)
    fine = g.standard_normal((64, 128))
    c = qtt.grid_restrict(ctx, fine, 3)
    ref = N.restrict(fine, 3)
    assert c.shape == (8, 16)
    assert np.allclose(c, ref, rtol=1e-6, atol=1e-6)
    coarse = g.standard_normal((8, 16)).astype(np.float32)
    f = qtt.grid_prolong(ctx, coarse, 3)
    assert f.shape == (64, 128)
    assert rel(f, N.prolong(coarse.astype(np.float64), 3)) < 1e-15
    assert rel(qtt.grid_prolong(ctx, coarse, 0), coarse) == 0.0
    m, r = qtt.field_moments(ctx, coarse)
    assert abs(m - coarse.astype(np.float64).mean()) < 1e-12
    assert abs(r - np.sqrt((coarse.astype(np.float64) ** 2).mean())) < 1e-12
