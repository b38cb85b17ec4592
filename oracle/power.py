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

Redshift-space multipoles (the paper's RSD study, Eq. 5; not a step of the
COLA loop): particles are moved along the line of sight z by their peculiar
velocity, s = x + z_hat p_z / (a^2 E(a)) in the code units (t in 1/H0,
p = a^2 dx/dt), with the full momentum p = v + a^3 E(a) [D1'(a) Psi1 +
D2'(a) Psi2] of the COLA state (p = v in the PM-only mode), and
P_l(k) = (2l + 1) <|delta_s(k)|^2 L_l(mu)> over the modes of each bin, mu = k_z/|k|.

Pins (tests/test_oracle_power.py): mode counts per bin against brute force;
a single injected mode lands in its bin with its amplitude; white noise has a
flat spectrum of the expected level; a plane wave along z or x gives the
Legendre values exactly; a small-amplitude Zel'dovich field obeys the Kaiser
limit delta_s(k) = (1 + f mu^2) delta(k).
"""
from __future__ import annotations

import numpy as np

from .cosmology import E
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


def legendre2(mu):
    return 0.5 * (3.0 * mu**2 - 1.0)


def legendre4(mu):
    return (35.0 * mu**4 - 30.0 * mu**2 + 3.0) / 8.0


def multipoles_from_delta(delta: np.ndarray, L: float, flags: int = 0):
    """Returns (k_mean, P0, P2, P4, n_modes) with P_l = (2l + 1) <P(k) L_l(mu)>,
    mu = n_z / |n|, over the bins of power_from_delta (the same weights,
    deconvolution and aliasing options)."""
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
        p = p / ((np.sinc(nx / ng) * np.sinc(ny / ng) * np.sinc(nz / ng)) ** 2) ** 2
    if flags & ALIAS_JING:
        s = lambda t: np.sin(np.pi * t / ng) ** 2
        p = p / ((1 - 2.0 / 3.0 * s(nx)) * (1 - 2.0 / 3.0 * s(ny)) * (1 - 2.0 / 3.0 * s(nz)))
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(n2 > 0, nz / np.sqrt(n2.astype(np.float64)), 0.0)
    kmag = 2.0 * np.pi / L * np.sqrt(n2.astype(np.float64))
    i = np.floor(np.sqrt(n2.astype(np.float64)) + 0.5).astype(np.int64)
    sel = (n2 > 0) & (i >= 1) & (i <= nb)
    ib = i[sel] - 1
    ws = w[sel]
    ps = p[sel]
    ms = mu[sel]
    nmodes = np.bincount(ib, weights=ws, minlength=nb)
    ksum = np.bincount(ib, weights=ws * kmag[sel], minlength=nb)
    out = [np.bincount(ib, weights=ws * ps * leg, minlength=nb) * (2 * l + 1)
           for l, leg in ((0, 1.0), (2, legendre2(ms)), (4, legendre4(ms)))]
    with np.errstate(invalid="ignore", divide="ignore"):
        return (ksum / nmodes, out[0] / nmodes, out[1] / nmodes, out[2] / nmodes, nmodes)


def redshift_space_displacement(state: dict, a: float, D1p: float, D2p: float, c, pm_only: bool = False):
    """Displacement of the particles in redshift space along z at scale factor
    a: d + z_hat p_z / (a^2 E(a)), p = v + a^3 E(a) (D1'(a) Psi1 + D2'(a) Psi2)
    (D' = dD/da; p = v in the PM-only mode)."""
    Ea = float(E(a, c))
    pz = state["v"][2].astype(np.float64)
    if not pm_only:
        pz = pz + a**3 * Ea * (D1p * state["psi1"][2] + D2p * state["psi2"][2])
    out = np.array(state["d"], dtype=np.float64, copy=True)
    out[2] += pz / (a * a * Ea)
    return out


def power_multipoles(d, nq: int, ng_pk: int, L: float, flags: int = 0):
    """Multipoles of a (redshift-space) displacement field d (3, Np) on an ng_pk^3 CIC mesh."""
    return multipoles_from_delta(density_contrast(d, nq, ng_pk, L), L, flags)
