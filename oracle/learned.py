"""FP64 forward and backward of the learned coarse-mesh force correction.

Test infrastructure only (see ``oracle/__init__``).

The paper has no learned component; this is the correction the build adds on
the PM_grid = 1 mesh (the paper finds coarser force meshes biased: PM_grid = 2
against 3 moves the matter P(k) by about 1 % and the halo abundance more, Sec. 4.4).
Definitions, shared by the CUDA path (which rounds weights and activations to
BF16 and accumulates in FP32):

* conv(x, W, b)[o, v] = b[o] + sum_{c, t} W[o, c, t] x[c, v + t - 1], with
  t = (tx, ty, tz) in {0,1,2}^3 and circular (periodic) indexing: a 3x3x3
  cross-correlation on the periodic mesh.
* net(x) = conv(relu(conv(relu(conv(x, W1, b1)), W2, b2)), W3, b3) with input
  channels (delta, F_x, F_y, F_z) and three output channels: the residual
  force added to the (filtered) coarse force mesh.
* Loss over particles: L = 1/(2 Np) sum_p |G(F + net)(p) - F_target(p)|^2,
  G the CIC gather; its adjoint is the CIC deposit of the residuals.

Pins (tests/test_oracle_learned.py): central finite differences of L with
respect to every parameter tensor and the input; a single-tap kernel is a
periodic shift (np.roll); linearity of the gather adjoint.
"""
from __future__ import annotations

import numpy as np

from .pm import cic_deposit, cic_gather

OFFSETS = [(tx, ty, tz) for tx in range(3) for ty in range(3) for tz in range(3)]


def shift(x: np.ndarray, t) -> np.ndarray:
    """s[..., v] = x[..., v + t - 1] on the periodic mesh (last three axes)."""
    return np.roll(x, shift=(1 - t[0], 1 - t[1], 1 - t[2]), axis=(-3, -2, -1))


def conv(x: np.ndarray, W: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x (C, N, N, N), W (O, C, 3, 3, 3), b (O,) -> (O, N, N, N)."""
    out = np.zeros((W.shape[0],) + x.shape[1:])
    for t in OFFSETS:
        xs = shift(x, t)
        out += np.einsum("oc,cxyz->oxyz", W[:, :, t[0], t[1], t[2]], xs)
    return out + b[:, None, None, None]


def conv_backward(dy: np.ndarray, x: np.ndarray, W: np.ndarray):
    """Gradients of sum(dy * conv(x, W, b)) w.r.t. x, W, b."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t in OFFSETS:
        xs = shift(x, t)
        dW[:, :, t[0], t[1], t[2]] = np.einsum("oxyz,cxyz->oc", dy, xs)
        # y[v] uses x[v + t - 1]: scatter back with the opposite shift
        g = np.einsum("oc,oxyz->cxyz", W[:, :, t[0], t[1], t[2]], dy)
        dx += np.roll(g, shift=(t[0] - 1, t[1] - 1, t[2] - 1), axis=(-3, -2, -1))
    db = dy.sum(axis=(1, 2, 3))
    return dx, dW, db


def net_forward(x: np.ndarray, p: dict):
    z1 = conv(x, p["W1"], p["b1"])
    h1 = np.maximum(z1, 0.0)
    z2 = conv(h1, p["W2"], p["b2"])
    h2 = np.maximum(z2, 0.0)
    out = conv(h2, p["W3"], p["b3"])
    return out, {"x": x, "z1": z1, "h1": h1, "z2": z2, "h2": h2}


def net_backward(dout: np.ndarray, cache: dict, p: dict):
    g = {}
    dh2, g["W3"], g["b3"] = conv_backward(dout, cache["h2"], p["W3"])
    dz2 = dh2 * (cache["z2"] > 0)
    dh1, g["W2"], g["b2"] = conv_backward(dz2, cache["h1"], p["W2"])
    dz1 = dh1 * (cache["z1"] > 0)
    g["x"], g["W1"], g["b1"] = conv_backward(dz1, cache["x"], p["W1"])
    return g


def particle_loss(mesh_force: np.ndarray, u: np.ndarray, target: np.ndarray):
    """L = 1/(2 Np) sum |G(mesh_force)(p) - target(p)|^2 and dL/dmesh_force
    (the CIC deposit of the residuals / Np)."""
    ng = mesh_force.shape[1]
    np_ = u.shape[1]
    pred = np.stack([cic_gather(mesh_force[j], u) for j in range(3)])
    res = pred - target
    loss = 0.5 * np.sum(res**2) / np_
    grad = np.stack([cic_deposit(u, ng, weights=res[j]) for j in range(3)]) / np_
    return loss, grad


def init_params(seed: int, cin=4, c=16, cout=3, scale=0.1):
    rng = np.random.default_rng(seed)
    def w(o, i):
        return rng.standard_normal((o, i, 3, 3, 3)) * scale / np.sqrt(27 * i)
    return {"W1": w(c, cin), "b1": np.zeros(c), "W2": w(c, c), "b2": np.zeros(c),
            "W3": w(cout, c), "b3": np.zeros(cout)}


def filter_row(a: float, nrows: int, a_init: float, a_final: float) -> int:
    """Row of a scale-factor-dependent filter table used at scale factor a:
    rows sit at a_r = a_init + r (a_final - a_init) / (nrows - 1) and the
    nearest one is used (a single row for nrows <= 1)."""
    if nrows <= 1:
        return 0
    nodes = a_init + np.arange(nrows) * (a_final - a_init) / (nrows - 1)
    return int(np.argmin(np.abs(nodes - a)))


def radial_bins(ng: int, L: float, nbins: int):
    """Piecewise-linear hat basis in |k| for the k-space filter: node b at
    k_b = b * k_max / (nbins - 1), k_max = sqrt(3) pi ng / L."""
    kmax = np.sqrt(3.0) * np.pi * ng / L
    return np.linspace(0.0, kmax, nbins)
