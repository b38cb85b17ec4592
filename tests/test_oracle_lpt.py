"""Pins of oracle/lpt.py: closed-form plane waves and the noise normalisation."""
import numpy as np

from oracle import cosmology as cm
from oracle import lpt, power
from oracle.philox import white_noise_grid
from synth import crossed_waves_delta


def _dk(delta):
    return np.fft.rfftn(delta)


def test_plane_wave_zeldovich_and_no_second_order():
    n, L, A = 16, 100.0, 0.3
    k = 2 * np.pi / L
    delta = crossed_waves_delta(n, L, A, 0.0)
    psi1, psi2, delta2 = lpt.lpt_from_delta_k(_dk(delta), L)
    x = np.arange(n) * L / n
    np.testing.assert_allclose(psi1[0], np.broadcast_to((-(A / k) * np.sin(k * x))[:, None, None], (n, n, n)), atol=1e-12)
    assert np.abs(psi1[1:]).max() < 1e-13
    assert np.abs(psi2).max() < 1e-13 and np.abs(delta2).max() < 1e-13


def test_crossed_waves_second_order_closed_form():
    n, L, A, B = 16, 64.0, 0.2, -0.35
    k = 2 * np.pi / L
    psi1, psi2, delta2 = lpt.lpt_from_delta_k(_dk(crossed_waves_delta(n, L, A, B)), L)
    x = np.arange(n) * L / n
    cx, sx = np.cos(k * x)[:, None, None], np.sin(k * x)[:, None, None]
    cy, sy = np.cos(k * x)[None, :, None], np.sin(k * x)[None, :, None]
    np.testing.assert_allclose(delta2, np.broadcast_to(A * B * cx * cy, (n, n, n)), atol=1e-12)
    np.testing.assert_allclose(psi2[0], np.broadcast_to(A * B / (2 * k) * sx * cy, (n, n, n)), atol=1e-12)
    np.testing.assert_allclose(psi2[1], np.broadcast_to(A * B / (2 * k) * cx * sy, (n, n, n)), atol=1e-12)
    assert np.abs(psi2[2]).max() < 1e-13


def test_divergence_of_psi1_is_minus_delta():
    # band-limited random field: finite-difference divergence of a smooth Psi1
    n, L = 32, 32.0
    rng = np.random.default_rng(4)
    dk = np.fft.rfftn(rng.standard_normal((n, n, n)))
    kx, ky, kz, *_ = lpt.kgrid(n, L)
    dk = np.where(kx**2 + ky**2 + kz**2 > (2 * np.pi / L * 3) ** 2, 0.0, dk)
    psi1, _, _ = lpt.lpt_from_delta_k(dk, L)
    delta = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2))
    h = L / n
    div = sum((np.roll(psi1[i], -1, i) - np.roll(psi1[i], 1, i)) / (2 * h) for i in range(3))
    # central differences are O(h^2 k^2) accurate for k <= 3 k_F
    assert np.abs(div + delta).max() < 0.1 * np.abs(delta).max()


def test_noise_field_power_matches_linear_spectrum():
    c = cm.Cosmology()
    P = cm.LinearPower(c)
    n, L = 64, 256.0
    dk = lpt.linear_delta_k(white_noise_grid(3, n), L, P)
    delta = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2))
    k, p, nm = power.power_from_delta(delta, L)
    sel = slice(4, 24)
    ratio = p[sel] / P(k[sel])
    # cosmic variance per bin ~ sqrt(2/N_modes) ~ 2-6 %; the mean over 20 bins ~ 1 %
    assert abs(ratio.mean() - 1.0) < 0.03
    assert np.all(np.abs(ratio - 1) < 5 * np.sqrt(2 / nm[sel]) + 0.02)
    # Nyquist modes removed, mean removed
    assert abs(delta.mean()) < 1e-14
    assert np.all(dk[n // 2, :, :] == 0) and np.all(dk[:, :, n // 2] == 0)
