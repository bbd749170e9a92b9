"""Pins of the FP64 MLP reference: torch float64 autograd, finite differences, torch Adam."""
import math

import numpy as np
import pytest
import torch

import synth
from oracle import mlp as M


def _torch_net(theta):
    layers = M.unflatten(theta)
    ts = [(torch.tensor(w, dtype=torch.float64, requires_grad=True),
           torch.tensor(b, dtype=torch.float64, requires_grad=True)) for w, b in layers]
    return ts


def _torch_forward(ts, x):
    h = torch.tensor(x, dtype=torch.float64)
    for li, (w, b) in enumerate(ts):
        h = h @ w.T + b
        if li < len(ts) - 1:
            h = torch.nn.functional.gelu(h, approximate="none")
    return h[:, 0]


def _batch(seed=61, nb=16):
    g = np.random.Generator(np.random.PCG64(seed))
    x = np.concatenate([g.dirichlet(np.ones(64), nb), g.uniform(-7, -3, (nb, 1))], axis=1)
    y = g.uniform(-12, -2, nb)
    return x, y


def test_forward_and_backward_match_torch_autograd():
    theta = synth.mlp_init(7).astype(np.float64)
    x, y = _batch()
    q = 0.1
    loss, grad = M.loss_and_grad(theta, x, y, q)
    ts = _torch_net(theta)
    yp = _torch_forward(ts, x)
    r = torch.tensor(y) - yp
    tl = torch.mean(torch.maximum(q * r, (q - 1) * r))
    tl.backward()
    tg = np.concatenate([np.concatenate([w.grad.numpy().ravel(), b.grad.numpy().ravel()])
                         for w, b in ts])
    assert math.isclose(loss, tl.item(), rel_tol=1e-13)
    assert np.allclose(M.forward(theta, x)[0], yp.detach().numpy(), rtol=1e-13, atol=1e-15)
    assert np.allclose(grad, tg, rtol=1e-11, atol=1e-15)


def test_backward_matches_central_differences():
    theta = synth.mlp_init(8).astype(np.float64)
    x, _ = _batch(62, 4)
    dy = np.array([0.3, -1.1, 0.7, 2.0])

    def f(t):
        return float(np.dot(dy, M.forward(t, x)[0]))

    _, cache = M.forward(theta, x)
    g = M.backward(theta, cache, dy)
    g_fd = M.finite_difference_grad(f, theta, 1e-6)
    assert np.max(np.abs(g - g_fd)) <= 1e-6 * max(1.0, np.max(np.abs(g)))


def test_one_hidden_unit_by_hand():
    """sizes (1,1,1,1): y = w3 gelu(w2 gelu(w1 x + b1) + b2) + b3 with gelu(0) = 0, gelu(z) ~ z for z >> 0."""
    sizes = (1, 1, 1, 1)
    theta = np.array([2.0, -1.0, 1.0, 0.0, 3.0, 0.5])   # w1 b1 w2 b2 w3 b3
    y, _ = M.forward(theta, np.array([[0.5]]), sizes)        # z1 = 0 -> h1 = 0 -> z2 = 0 -> y = b3
    assert y[0] == 0.5
    y, cache = M.forward(theta, np.array([[20.0]]), sizes)   # z1 = 39 -> h1 = 39 -> y = 3*39 + 0.5
    assert y[0] == 117.5
    g = M.backward(theta, cache, np.array([1.0]), sizes)
    # dy/dw3 = h2 = 39; dy/db3 = 1; dy/dw2 = w3 * h1 = 117; dy/dw1 = w3 w2 x = 60
    assert np.allclose(g[[4, 5, 2, 0]], [39.0, 1.0, 117.0, 60.0], rtol=1e-12)


def test_adam_matches_torch():
    theta = synth.mlp_init(9).astype(np.float64)
    x, y = _batch(63, 8)
    m = np.zeros_like(theta)
    v = np.zeros_like(theta)
    tt = torch.tensor(theta.copy(), requires_grad=True)
    opt = torch.optim.Adam([tt], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    th = theta.copy()
    for step in range(1, 4):
        _, g = M.loss_and_grad(th, x, y, 0.2)
        th, m, v = M.adam_step(th, g, m, v, step, 1e-3)
        opt.zero_grad()
        _, g2 = M.loss_and_grad(tt.detach().numpy().copy(), x, y, 0.2)
        tt.grad = torch.tensor(g2)
        opt.step()
    assert np.allclose(th, tt.detach().numpy(), rtol=1e-12, atol=1e-14)


def test_pinball_loss_by_hand_and_quantile_minimiser():
    """rho_q(r) = q r for r > 0 and (q - 1) r otherwise, checked on hand values; a constant
    prediction minimising the mean loss is a q-quantile of the targets (the textbook property
    the learned tau relies on); the gradient matches central differences away from kinks."""
    q = 0.8
    assert M.pinball_loss([0.0, 0.0], [2.0, -1.0], q) == pytest.approx((0.8 * 2 + 0.2 * 1) / 2)
    g = np.random.Generator(np.random.PCG64(64))
    y = g.normal(size=101)
    grid = np.linspace(-3, 3, 6001)
    losses = [M.pinball_loss(np.full_like(y, c), y, q) for c in grid]
    best = grid[int(np.argmin(losses))]
    ys = np.sort(y)
    assert ys[79] - 1e-3 <= best <= ys[81] + 1e-3          # the 0.8-quantile of 101 values
    pred = g.normal(size=7)
    tgt = g.normal(size=7)
    grad = M.pinball_grad(pred, tgt, q)
    h = 1e-6
    for t in range(7):
        up, dn = pred.copy(), pred.copy()
        up[t] += h
        dn[t] -= h
        fd = (M.pinball_loss(up, tgt, q) - M.pinball_loss(dn, tgt, q)) / (2 * h)
        assert grad[t] == pytest.approx(fd, rel=1e-6, abs=1e-9)
