"""Linear density field and 2LPT displacements (Sec. 2.2: Gaussian initial
conditions with 2LPT, Crocce, Pueblas & Scoccimarro 2006).

Test infrastructure only (see ``oracle/__init__``).

Readings (the paper prints no formula for this step):

* Lagrangian grid q_n = n * dq, dq = L/nq, no offset; particle index
  p = (i*nq + j)*nq + k (C order, z fastest).
* delta_k = FFT(w) * sqrt(P_lin(k) / dq^3): with an unnormalised forward DFT,
  <|w_k|^2> = nq^3, so <|delta_k|^2> = nq^6 P / L^3, the discrete image of P.
  k = 2 pi n / L with signed n; the k=0 mode and every mode with any
  |n_i| = nq/2 (Nyquist) are set to zero so that all derived fields are real.
* First order: Psi1 = -grad phi1, lap phi1 = delta  =>  Psi1_k = i k delta_k / k^2
  (div Psi1 = -delta).
* Second order: delta2 = sum_{i<j} [phi1_ii phi1_jj - phi1_ij^2] in real space,
  Psi2 = +grad phi2 with lap phi2 = delta2  =>  Psi2_k = -i k delta2_k / k^2.
* Positions x = q + D1 Psi1 + D2 Psi2 with D2 ~ -3/7 D1^2 (D1(1)=1, so delta is
  the linear field extrapolated to a=1).

Pins (tests/test_oracle_lpt.py): a single plane wave has the closed-form
Zel'dovich displacement and Psi2 = 0; two crossed waves A cos kx + B cos ky give
delta2 = AB cos kx cos ky and Psi2 = (AB/2k)(sin kx cos ky, cos kx sin ky, 0);
div Psi1 = -delta; the noise power matches P(k) on average.
"""
from __future__ import annotations

import numpy as np

from .philox import white_noise_grid

# FFT backend of the 2LPT and PM transforms: numpy.fft (pocketfft), or
# scipy.fft's pocketfft with worker threads when FFT_WORKERS > 1 (same
# algorithm; used for full-size references and the timed CPU baseline)
FFT_WORKERS = 1


def _rfftn(x):
    if FFT_WORKERS > 1:
        import scipy.fft
        return scipy.fft.rfftn(x, workers=FFT_WORKERS)
    return np.fft.rfftn(x)


def _irfftn(x, shape):
    if FFT_WORKERS > 1:
        import scipy.fft
        return scipy.fft.irfftn(x, s=shape, axes=(0, 1, 2), workers=FFT_WORKERS)
    return np.fft.irfftn(x, s=shape, axes=(0, 1, 2))


def kgrid(n: int, L: float):
    """Signed wavenumbers (kx, ky) on the full axes and kz on the half axis,
    plus the Nyquist masks, for an n^3 mesh of side L."""
    nfull = np.fft.fftfreq(n, d=1.0 / n)           # 0..n/2-1, -n/2..-1
    nhalf = np.arange(n // 2 + 1, dtype=np.float64)
    kf = 2.0 * np.pi / L
    kx = (kf * nfull)[:, None, None]
    ky = (kf * nfull)[None, :, None]
    kz = (kf * nhalf)[None, None, :]
    nyq_x = (np.abs(nfull) == n // 2)[:, None, None]
    nyq_y = (np.abs(nfull) == n // 2)[None, :, None]
    nyq_z = (nhalf == n // 2)[None, None, :]
    return kx, ky, kz, nyq_x, nyq_y, nyq_z


def linear_delta_k(noise: np.ndarray, L: float, pk) -> np.ndarray:
    """delta_k = FFT(noise) sqrt(P(k)/dq^3), with k=0 and Nyquist modes zeroed."""
    n = noise.shape[0]
    kx, ky, kz, nx, ny, nz = kgrid(n, L)
    k = np.sqrt(kx**2 + ky**2 + kz**2)
    dq3 = (L / n) ** 3
    wk = _rfftn(noise)
    dk = wk * np.sqrt(pk(k) / dq3)
    dk = np.where(nx | ny | nz, 0.0, dk)
    dk[0, 0, 0] = 0.0
    return dk


def lpt_from_delta_k(dk: np.ndarray, L: float):
    """(Psi1, Psi2), each of shape (3, n, n, n), from the linear delta_k (a=1).
    Also returns delta2 for inspection."""
    n = dk.shape[0]
    kx, ky, kz, nx, ny, nz = kgrid(n, L)
    kv = [kx, ky, kz]
    k2 = kx**2 + ky**2 + kz**2
    k2[0, 0, 0] = 1.0
    shape = (n, n, n)
    psi1 = np.stack([_irfftn(1j * kv[i] * dk / k2, shape) for i in range(3)])
    # phi1_ij = IFFT[ -k_i k_j phi1_k ] = IFFT[ k_i k_j delta_k / k^2 ]
    phi = {}
    for i in range(3):
        for j in range(i, 3):
            phi[i, j] = _irfftn(kv[i] * kv[j] * dk / k2, shape)
    delta2 = (phi[0, 0] * phi[1, 1] + phi[0, 0] * phi[2, 2] + phi[1, 1] * phi[2, 2]
              - phi[0, 1] ** 2 - phi[0, 2] ** 2 - phi[1, 2] ** 2)
    d2k = _rfftn(delta2)
    d2k = np.where(nx | ny | nz, 0.0, d2k)
    d2k[0, 0, 0] = 0.0
    psi2 = np.stack([_irfftn(-1j * kv[i] * d2k / k2, shape) for i in range(3)])
    return psi1, psi2, delta2


def initial_conditions(seed: int, nq: int, L: float, pk, D1_init: float, D2_init: float):
    """2LPT initial state.  Returns dict with psi1, psi2 of shape (3, nq^3)
    (particle order = C order of the Lagrangian grid), the displacement
    d = D1 Psi1 + D2 Psi2 and the residual momentum v = 0."""
    noise = white_noise_grid(seed, nq)
    dk = linear_delta_k(noise, L, pk)
    psi1, psi2, _ = lpt_from_delta_k(dk, L)
    psi1 = psi1.reshape(3, -1)
    psi2 = psi2.reshape(3, -1)
    return {
        "psi1": psi1,
        "psi2": psi2,
        "d": D1_init * psi1 + D2_init * psi2,
        "v": np.zeros_like(psi1),
    }
