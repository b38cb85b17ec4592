"""Matter power spectrum estimator (Sec. 2.5: CIC assignment to a mesh, FFT,
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
* flags & 4 (ALIAS_ITER): the full Jing (2005) correction of the CIC window and its
  aliases, iterated.  Each mode's raw power is modelled as
  C(m) P(|m|), C(m) = sum over images n in [-2, 2]^3 of W^2(m + ng n)
  (|m + ng n| / |m|)^n_eff, W the CIC window (a product over axes of
  sinc^2(pi x / ng)), i.e. P locally a power law of index n_eff around |m|.
  sin(pi (m + ng n) / ng) = +-sin(pi m / ng), so each image's window factor is
  sin^4(pi m_i / ng) / (pi (m_i + ng n_i) / ng)^4 per axis (1 for m_i = n_i = 0,
  0 for m_i = 0 != n_i).  The estimate starts from the closed-form one (flags 1 | 2);
  each of three iterations takes n_eff per bin as the log-slope of the previous
  estimate between the neighbouring bins (one-sided at the ends, 0 where a power is
  not positive, clamped to [-4, 4]) and sets P(bin) = < raw / C >.  Replaces flags 1
  and 2.  The number of images, the slope rule and the iteration count are readings:
  Jing (2005) gives the model and the iteration, the paper only cites it.

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

import itertools

import numpy as np

from .cosmology import E
from .pm import density_contrast

DECONV_CIC = 1
ALIAS_JING = 2
ALIAS_ITER = 4
JING_IMAGES = 2
JING_ITERATIONS = 3
NEFF_CLAMP = 4.0


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


def _modes(ng: int):
    nfull = np.fft.fftfreq(ng, d=1.0 / ng).astype(np.int64)
    nhalf = np.arange(ng // 2 + 1, dtype=np.int64)
    return nfull[:, None, None], nfull[None, :, None], nhalf[None, None, :]


def jing_alias_sum(nx, ny, nz, ng: int, neff, images: int = JING_IMAGES):
    """C(m) = sum_{n in [-J, J]^3} W^2(m + ng n) (|m + ng n| / |m|)^neff for the
    integer mode vectors (nx, ny, nz) (broadcast arrays), W the CIC window."""
    m = [np.asarray(x, dtype=np.float64) for x in (nx, ny, nz)]
    m2 = m[0] ** 2 + m[1] ** 2 + m[2] ** 2
    neff = np.asarray(neff, dtype=np.float64)
    s4 = [np.sin(np.pi * x / ng) ** 4 for x in m]
    total = 0.0
    for n in itertools.product(range(-images, images + 1), repeat=3):
        w = 1.0
        r2 = 0.0
        for a in range(3):
            x = m[a] + ng * n[a]
            with np.errstate(divide="ignore", invalid="ignore"):
                fa = np.where(m[a] == 0, 1.0 if n[a] == 0 else 0.0, s4[a] / (np.pi * x / ng) ** 4)
            w = w * fa
            r2 = r2 + x * x
        with np.errstate(divide="ignore", invalid="ignore"):
            ratio = np.where(m2 > 0, r2 / np.where(m2 > 0, m2, 1.0), 1.0)
        total = total + w * ratio ** (0.5 * neff)
    return total


def local_slopes(k: np.ndarray, p: np.ndarray) -> np.ndarray:
    """n_eff per bin: d ln P / d ln k from the neighbouring bins (one-sided at the
    ends; 0 where a power is not positive), clamped to [-NEFF_CLAMP, NEFF_CLAMP]."""
    nb = len(p)
    out = np.zeros(nb)
    for b in range(nb):
        lo, hi = max(b - 1, 0), min(b + 1, nb - 1)
        if hi == lo or not (p[lo] > 0 and p[hi] > 0 and k[hi] > k[lo] > 0):
            continue
        out[b] = np.clip(np.log(p[hi] / p[lo]) / np.log(k[hi] / k[lo]), -NEFF_CLAMP, NEFF_CLAMP)
    return out


def power_jing_iterative(delta: np.ndarray, L: float):
    """(k_mean, P, n_modes) with the iterated Jing (2005) correction (flags 4)."""
    ng = delta.shape[0]
    nb = ng // 2
    k, p, nm = power_from_delta(delta, L, DECONV_CIC | ALIAS_JING)
    dk = np.fft.rfftn(delta)
    praw = np.abs(dk) ** 2 * L**3 / float(ng) ** 6
    nx, ny, nz = _modes(ng)
    n2 = nx**2 + ny**2 + nz**2
    w = np.where((nz == 0) | (nz == ng // 2), 1.0, 2.0) * np.ones_like(n2, dtype=np.float64)
    i = np.floor(np.sqrt(n2.astype(np.float64)) + 0.5).astype(np.int64)
    sel = (n2 > 0) & (i >= 1) & (i <= nb)
    ib = np.where(sel, i - 1, 0)
    for _ in range(JING_ITERATIONS):
        neff = local_slopes(k, p)[ib]
        C = jing_alias_sum(nx, ny, nz, ng, neff)
        q = np.where(sel, praw / np.where(sel, C, 1.0), 0.0)
        with np.errstate(invalid="ignore", divide="ignore"):
            p = np.bincount(ib[sel], weights=(w * q)[sel], minlength=nb) / nm
    return k, p, nm


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
