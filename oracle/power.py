"""Matter power spectrum estimator (Sec. 2.4: CIC assignment to a mesh, FFT,
band power P(k) = <|delta_k|^2> over the modes of a k-bin, CIC deconvolution,
Jing 2005 aliasing correction).

Test infrastructure only (see ``oracle/__init__``).

Readings:
* P(k_n) = |delta_k|^2 L^3 / ng^6 with the unnormalised forward DFT.
* Bin i (i = 1 .. ng/2) holds the modes with integer |n|^2 in
  [i^2 - i + 1, i^2 + i], i.e. (i - 1/2) < |n| < (i + 1/2): shells one
  fundamental mode wide centred on i k_F, decided in integer arithmetic.
* Sums run over the full k-space: half-spectrum modes count twice except on
  the k_z = 0 and k_z = Nyquist planes.  k_mean is the mode-weighted mean |k|.
* flags & 1 (DECONV_CIC): divide each mode by W^2, W = prod_i sinc^2(pi n_i/ng).
* flags & 2 (ALIAS_JING): divide each mode by prod_i [1 - 2/3 sin^2(pi n_i/ng)],
  the closed-form CIC alias sum for a shot-noise dominated field (Jing 2005).
  The paper cites Jing 2005 without detail; this closed form is the reading.
* No shot-noise subtraction for matter (the paper applies it to halo monopoles).

Pins (tests/test_oracle_power.py): mode counts per bin against brute force;
a single injected mode lands in its bin with its amplitude; white noise has a
flat spectrum of the expected level.
"""
from __future__ import annotations

import numpy as np

from .pm import density_contrast

DECONV_CIC = 1
ALIAS_JING = 2


def power_from_delta(delta: np.ndarray, L: float, flags: int = 0):
    """Returns (k_mean, P, n_modes) for bins i = 1 .. ng/2 (index i-1)."""
    ng = delta.shape[0]
    nb = ng // 2
    dk = np.fft.rfftn(delta)
    nfull = np.fft.fftfreq(ng, d=1.0 / ng).astype(np.int64)
    nhalf = np.arange(ng // 2 + 1, dtype=np.int64)
    nx = nfull[:, None, None]
    ny = nfull[None, :, None]
    nz = nhalf[None, None, :]
    n2 = nx**2 + ny**2 + nz**2
    w = np.where((nz == 0) | (nz == ng // 2), 1.0, 2.0) * np.ones_like(n2, dtype=np.float64)
    p = np.abs(dk) ** 2 * L**3 / float(ng) ** 6
    if flags & DECONV_CIC:
        W = (np.sinc(nx / ng) * np.sinc(ny / ng) * np.sinc(nz / ng)) ** 2  # np.sinc(x)=sin(pi x)/(pi x)
        p = p / W**2
    if flags & ALIAS_JING:
        s = lambda t: np.sin(np.pi * t / ng) ** 2
        p = p / ((1 - 2.0 / 3.0 * s(nx)) * (1 - 2.0 / 3.0 * s(ny)) * (1 - 2.0 / 3.0 * s(nz)))
    kmag = 2.0 * np.pi / L * np.sqrt(n2.astype(np.float64))
    # bin index: smallest i with n2 <= i^2 + i  <=>  i = round(sqrt(n2)) (no ties)
    i = np.floor(np.sqrt(n2.astype(np.float64)) + 0.5).astype(np.int64)
    i = np.broadcast_to(i, n2.shape)
    sel = (n2 > 0) & (i >= 1) & (i <= nb)
    ib = i[sel] - 1
    ws = np.broadcast_to(w, n2.shape)[sel]
    nmodes = np.bincount(ib, weights=ws, minlength=nb)
    psum = np.bincount(ib, weights=ws * np.broadcast_to(p, n2.shape)[sel], minlength=nb)
    ksum = np.bincount(ib, weights=ws * np.broadcast_to(kmag, n2.shape)[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        return ksum / nmodes, psum / nmodes, nmodes


def bin_of(n2: int) -> int:
    """Bin index (1-based) of an integer |n|^2 by the defining inequality."""
    i = 1
    while not (i * i - i + 1 <= n2 <= i * i + i):
        i += 1
    return i


def power_spectrum(d, nq: int, ng_pk: int, L: float, flags: int = 0):
    """P(k) of a particle displacement field d (3, Np) on an ng_pk^3 CIC mesh."""
    return power_from_delta(density_contrast(d, nq, ng_pk, L), L, flags)
