"""Pins of oracle/learned.py: finite differences of the hand backward,
single-tap kernels as periodic shifts, gather adjointness."""
import numpy as np
import pytest

from oracle import learned as ol
from oracle import pm


def test_single_tap_kernel_is_a_periodic_shift():
    rng = np.random.default_rng(0)
    x = rng.standard_normal((2, 5, 6, 7))
    for t in [(0, 1, 1), (2, 2, 0), (1, 1, 1)]:
        W = np.zeros((2, 2, 3, 3, 3))
        W[0, 1][t] = 1.0
        W[1, 0][t] = 2.0
        y = ol.conv(x, W, np.array([0.5, -1.0]))
        # y[v] = x[v + t - 1]
        ref0 = np.roll(x[1], shift=(1 - t[0], 1 - t[1], 1 - t[2]), axis=(0, 1, 2)) + 0.5
        np.testing.assert_allclose(y[0], ref0, atol=1e-14)
        i, j, k = 2, 3, 4
        assert y[1, i, j, k] == pytest.approx(2 * x[0, (i + t[0] - 1) % 5, (j + t[1] - 1) % 6, (k + t[2] - 1) % 7] - 1)


def _loss(p, x, u, base, target):
    out, cache = ol.net_forward(x, p)
    loss, grad = ol.particle_loss(base + out, u, target)
    return loss, grad, cache


def test_net_backward_matches_finite_differences():
    rng = np.random.default_rng(3)
    n, cin, c = 5, 4, 3
    p = ol.init_params(1, cin=cin, c=c, scale=1.0)
    for k in ("b1", "b2", "b3"):
        p[k] = rng.standard_normal(p[k].shape) * 0.1
    x = rng.standard_normal((cin, n, n, n))
    base = rng.standard_normal((3, n, n, n))
    u = rng.uniform(0, n, (3, 40))
    target = rng.standard_normal((3, 40))
    loss, dmesh, cache = _loss(p, x, u, base, target)
    g = ol.net_backward(dmesh, cache, p)
    h = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3", "x"):
        arr = x if name == "x" else p[name]
        flat = arr.reshape(-1)
        idx = rng.choice(flat.size, size=min(12, flat.size), replace=False)
        for i in idx:
            old = flat[i]
            flat[i] = old + h
            lp = _loss(p, x, u, base, target)[0]
            flat[i] = old - h
            lm = _loss(p, x, u, base, target)[0]
            flat[i] = old
            fd = (lp - lm) / (2 * h)
            an = g[name].reshape(-1)[i]
            assert an == pytest.approx(fd, rel=1e-6, abs=1e-9), (name, i)


def test_gather_adjoint_is_deposit():
    rng = np.random.default_rng(5)
    ng = 6
    u = rng.uniform(0, ng, (3, 30))
    f = rng.standard_normal((ng, ng, ng))
    w = rng.standard_normal(30)
    lhs = np.dot(pm.cic_gather(f, u), w)
    rhs = np.sum(f * pm.cic_deposit(u, ng, weights=w))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_filter_row_is_the_nearest_scale_factor_node():
    # rows at a = 0.05, 0.2875, 0.525, 0.7625, 1.0 (five nodes)
    assert ol.filter_row(0.05, 5, 0.05, 1.0) == 0
    assert ol.filter_row(1.0, 5, 0.05, 1.0) == 4
    assert ol.filter_row(0.16, 5, 0.05, 1.0) == 0
    assert ol.filter_row(0.17, 5, 0.05, 1.0) == 1
    assert ol.filter_row(0.6, 5, 0.05, 1.0) == 2
    assert ol.filter_row(0.01, 5, 0.05, 1.0) == 0
    assert ol.filter_row(0.7, 1, 0.05, 1.0) == 0
