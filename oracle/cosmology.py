"""Background cosmology, linear power spectrum, growth factors and the COLA time
integrals, in float64.

Test infrastructure only (see ``oracle/__init__``).

Conventions (the paper prints none of these; they are the readings the whole
oracle uses):

* Flat LCDM with the MICE parameters of Sec. 2.1 (Om=0.25, OL=0.75, Ob=0.044,
  ns=0.95, sigma8=0.8, h=0.7).  Lengths in Mpc/h, time in units of 1/H0, so
  H(a) = E(a) = sqrt(Om a^-3 + Ok a^-2 + OL).
* Linear P(k) = A k^ns T(k)^2 with T the Eisenstein & Hu (1998) no-wiggle
  ("zero baryon, Gamma_eff") fit, normalised to sigma8 at a=1.  The paper used
  CAMB (Sec. 2.1), which is not available; the closed form stands in for it.
* Growth: D1 is the growing mode normalised to D1(1)=1; D2 solves the
  second-order growth equation with D2 -> -(3/7) D1^2 at early times (the
  2LPT convention of Crocce et al. 2006, cited in Sec. 2.2).
* COLA kick and drift integrals (Eq. 2 discretised on the left-hand side):
  with p = a^2 dx/dt, dp/da = F/(a E) and dx/da = p/(a^3 E), so
  K(a,b) = int_a^b da/(a E) and Dr(a,b) = int_a^b da/(a^3 E).
* Time nodes: Eq. 3, n nodes with constant Delta f(a) = (f(a_f)-f(a_i))/(n-1).

Pins (tests/test_oracle_cosmology.py): EdS closed forms of D1, D2, K, Dr;
Heath integral vs ODE for D1; D2/(-3/7 D1^2) -> 1 early and the
Bouchet et al. Om^(-1/143) fit; the top-hat sigma_R of a flat spectrum
(closed form 3A/(4 pi R^3)); T(k->0)=1; the paper's worked time-node example
(10 steps from a_i = step width gives z_i = 9, Sec. 4.3).
The EH98 fit constants themselves are parity unpinned beyond T(0)=1 and the
large-k asymptote (no tabulated values are available to compare against).
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np
from scipy import integrate


@dataclasses.dataclass(frozen=True)
class Cosmology:
    """Cosmological parameters (Sec. 2.1: the MICE-GC model)."""

    omega_m: float = 0.25
    omega_l: float = 0.75
    omega_b: float = 0.044
    h: float = 0.7
    sigma8: float = 0.8
    n_s: float = 0.95
    t_cmb: float = 2.7255

    @property
    def omega_k(self) -> float:
        return 1.0 - self.omega_m - self.omega_l


# ----------------------------------------------------------------------------
# background
# ----------------------------------------------------------------------------

def E(a, c: Cosmology):
    """H(a)/H0 for matter + curvature + Lambda."""
    a = np.asarray(a, dtype=np.float64)
    return np.sqrt(c.omega_m / a**3 + c.omega_k / a**2 + c.omega_l)


def dlnE_dlna(a, c: Cosmology):
    """d ln E / d ln a = (-3 Om a^-3 - 2 Ok a^-2) / (2 E^2)."""
    a = np.asarray(a, dtype=np.float64)
    return (-3.0 * c.omega_m / a**3 - 2.0 * c.omega_k / a**2) / (2.0 * E(a, c) ** 2)


def omega_m_of_a(a, c: Cosmology):
    a = np.asarray(a, dtype=np.float64)
    return c.omega_m / a**3 / E(a, c) ** 2


# ----------------------------------------------------------------------------
# linear power spectrum
# ----------------------------------------------------------------------------

def transfer_eh_nowiggle(k, c: Cosmology):
    """Eisenstein & Hu (1998, ApJ 496, 605) no-wiggle transfer function,
    their Eqs. 26 and 28-31; k in h/Mpc."""
    k = np.asarray(k, dtype=np.float64)
    om_h2 = c.omega_m * c.h**2
    ob_h2 = c.omega_b * c.h**2
    fb = c.omega_b / c.omega_m
    theta = c.t_cmb / 2.7
    # sound horizon fit (Eq. 26), Mpc (not Mpc/h)
    s = 44.5 * math.log(9.83 / om_h2) / math.sqrt(1.0 + 10.0 * ob_h2**0.75)
    # baryon suppression of the shape parameter (Eq. 31)
    alpha = 1.0 - 0.328 * math.log(431.0 * om_h2) * fb + 0.38 * math.log(22.3 * om_h2) * fb**2
    k_mpc = k * c.h
    gamma_eff = c.omega_m * c.h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k_mpc * s) ** 4))  # Eq. 30
    q = k * theta**2 / gamma_eff  # Eq. 28, k in h/Mpc
    L0 = np.log(2.0 * math.e + 1.8 * q)  # Eq. 29
    C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
    return L0 / (L0 + C0 * q**2)


def tophat_window(x):
    """Fourier transform of a unit-volume spherical top hat, W(0)=1."""
    x = np.asarray(x, dtype=np.float64)
    out = np.empty_like(x)
    small = np.abs(x) < 1e-3
    xs = x[small]
    out[small] = 1.0 - xs**2 / 10.0 + xs**4 / 280.0
    xl = x[~small]
    out[~small] = 3.0 * (np.sin(xl) - xl * np.cos(xl)) / xl**3
    return out


def sigma_R(pk, R: float, kmax: float | None = None) -> float:
    """sigma_R^2 = 1/(2 pi^2) int_0^kmax k^2 P(k) W(kR)^2 dk, integrated in ln k
    (kmax defaults to 2000/R, far in the k^(ns-4) tail of any CDM spectrum)."""

    def integrand(lnk):
        k = math.exp(lnk)
        return k**3 * float(pk(np.array([k]))[0]) * float(tophat_window(np.array([k * R]))[0]) ** 2

    # split the log range so the oscillating tail is resolved
    top = 2e3 / R if kmax is None else kmax
    edges = np.linspace(math.log(1e-7), math.log(top), 121)
    total = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        val, _ = integrate.quad(integrand, lo, hi, epsabs=0.0, epsrel=1e-11, limit=200)
        total += val
    return math.sqrt(total / (2.0 * math.pi**2))


class LinearPower:
    """P_lin(k, a=1) = A k^ns T(k)^2 normalised so that sigma_8 = c.sigma8."""

    def __init__(self, c: Cosmology):
        self.c = c
        self.amplitude = 1.0
        s8 = sigma_R(self, 8.0)
        self.amplitude = (c.sigma8 / s8) ** 2

    def __call__(self, k):
        k = np.asarray(k, dtype=np.float64)
        out = np.zeros_like(k)
        pos = k > 0
        out[pos] = self.amplitude * k[pos] ** self.c.n_s * transfer_eh_nowiggle(k[pos], self.c) ** 2
        return out


# ----------------------------------------------------------------------------
# growth
# ----------------------------------------------------------------------------

A_EARLY = 1e-5  # start of the growth integration; Om(a) = 1 to 1e-14 there


def _growth_rhs(lna, y, c: Cosmology):
    """y = (D1, dD1/dlna, D2, dD2/dlna).

    Linear growth:  D1'' + (2 + dlnE/dlna) D1' - 3/2 Om(a) D1 = 0
    Second order:   D2'' + (2 + dlnE/dlna) D2' - 3/2 Om(a) D2 = -3/2 Om(a) D1^2
    (' = d/dlna), i.e. D_tt + 2H D_t = 4 pi G rho D rewritten in ln a."""
    a = math.exp(lna)
    om = float(omega_m_of_a(a, c))
    fr = 2.0 + float(dlnE_dlna(a, c))
    D1, D1p, D2, D2p = y
    return [D1p, -fr * D1p + 1.5 * om * D1, D2p, -fr * D2p + 1.5 * om * (D2 - D1 * D1)]


class Growth:
    """D1, D2 and their a-derivatives from the growth ODEs, D1(1) = 1."""

    def __init__(self, c: Cosmology):
        self.c = c
        a0 = A_EARLY
        # Einstein-de Sitter growing modes at a0: D1 = a, D2 = -3/7 a^2
        y0 = [a0, a0, -3.0 / 7.0 * a0**2, -6.0 / 7.0 * a0**2]
        self._y0 = y0
        y1 = self._raw(np.array([1.0]))
        self._norm = y1[0, 0]

    def _raw(self, a):
        a = np.atleast_1d(np.asarray(a, dtype=np.float64))
        out = np.empty((a.size, 4))
        for i, ai in enumerate(a):
            sol = integrate.solve_ivp(
                _growth_rhs, (math.log(A_EARLY), math.log(ai)),
                self._y0, args=(self.c,), method="DOP853", rtol=1e-13, atol=1e-30)
            out[i] = sol.y[:, -1]
        return out

    def __call__(self, a):
        """Returns (D1, dD1/da, D2, dD2/da) at each a."""
        a = np.atleast_1d(np.asarray(a, dtype=np.float64))
        y = self._raw(a)
        n = self._norm
        D1 = y[:, 0] / n
        D2 = y[:, 2] / n**2
        dD1 = y[:, 1] / n / a
        dD2 = y[:, 3] / n**2 / a
        return D1, dD1, D2, dD2


def D1_heath(a, c: Cosmology):
    """Linear growth by the Heath (1977) integral, exact for matter + curvature
    + Lambda:  D1 propto E(a) int_0^a da' / (a' E(a'))^3, normalised D1(1)=1."""

    def g(x):
        val, _ = integrate.quad(lambda t: 1.0 / (t * float(E(t, c))) ** 3, 0.0, x,
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return float(E(x, c)) * val

    a = np.atleast_1d(np.asarray(a, dtype=np.float64))
    g1 = g(1.0)
    return np.array([g(x) / g1 for x in a])


# ----------------------------------------------------------------------------
# COLA time integrals and nodes
# ----------------------------------------------------------------------------

def kick_integral(a: float, b: float, c: Cosmology) -> float:
    """K(a,b) = int_a^b da / (a E(a))   (dp/da = F / (a E))."""
    val, _ = integrate.quad(lambda t: 1.0 / (t * float(E(t, c))), a, b, epsabs=0.0, epsrel=1e-13)
    return val


def drift_integral(a: float, b: float, c: Cosmology) -> float:
    """Dr(a,b) = int_a^b da / (a^3 E(a))   (dx/da = p / (a^3 E))."""
    val, _ = integrate.quad(lambda t: 1.0 / (t**3 * float(E(t, c))), a, b, epsabs=0.0, epsrel=1e-13)
    return val


# Modified kick and drift factors of Tassev, Zaldarriaga & Eisenstein (2013),
# the COLA paper the ICE-COLA paper cites for the method (Sec. 1, Eq. 2).
# With p = a^2 dx/dt, dx/da = p / (a^3 E) and dp/da = F / (a E):
# * the standard factors take F constant over a kick and p constant over a
#   drift (kick_integral, drift_integral);
# * the modified ones take the residual momentum to vary as a power of a,
#   a^n with n = n_LPT, about the reference time a_c at which the force, or
#   the momentum, is known:
#     kick:  p(a) = alpha + beta a^n with dp/da(a_c) = F(a_c) / (a_c E(a_c))
#            -> Delta p = F(a_c) (a_f^n - a_i^n) / (n a_c^n E(a_c))
#     drift: p(a) = p(a_c) (a / a_c)^n
#            -> Delta x = p(a_c) a_c^-n int_{a_i}^{a_f} a^n / (a^3 E) da
# n_LPT = -2.5 is the value that paper adopts.  The reading of their
# definitions in these variables is this module's.
N_LPT = -2.5


def kick_modified(a: float, b: float, ac: float, c: Cosmology, n: float = N_LPT) -> float:
    """Modified kick factor from a to b, reference time ac (force at ac)."""
    return (b**n - a**n) / (n * ac**n * float(E(ac, c)))


def drift_modified(a: float, b: float, ac: float, c: Cosmology, n: float = N_LPT) -> float:
    """Modified drift factor from a to b, reference time ac (momentum at ac)."""
    val, _ = integrate.quad(lambda t: t**n / (t**3 * float(E(t, c))), a, b, epsabs=0.0, epsrel=1e-13)
    return val / ac**n


def time_nodes(a_i: float, a_f: float, n: int, sampling="linear", p: float = 1.0):
    """Eq. 3: n nodes with constant Delta f = (f(a_f) - f(a_i)) / (n - 1).

    sampling: 'linear' (f = a), 'log' (f = ln a) or 'pow' (f = a^p)."""
    if n < 2:
        raise ValueError("need at least two nodes")
    j = np.arange(n, dtype=np.float64)
    if sampling == "linear":
        return a_i + j * (a_f - a_i) / (n - 1)
    if sampling == "log":
        return np.exp(math.log(a_i) + j * (math.log(a_f) - math.log(a_i)) / (n - 1))
    if sampling == "pow":
        f = a_i**p + j * (a_f**p - a_i**p) / (n - 1)
        return f ** (1.0 / p)
    raise ValueError(sampling)


@dataclasses.dataclass
class StepTable:
    """Per-node FP64 coefficients of the COLA kick-drift-kick loop.

    Node j (force evaluation at a_j):
      A_j  = F(x_j) - c1_j Psi1 - c2_j Psi2,
             c1 = 3/2 Om/a D1(a),  c2 = 3/2 Om/a (D2(a) - D1(a)^2)
      v   += kick_j A_j,  kick_j = K(a_{j-1/2}, a_j)[j>0] + K(a_j, a_{j+1/2})[j<n-1]
      d   += drift_j v + dD1_j Psi1 + dD2_j Psi2   (j < n-1 only)
    with a_{j+1/2} the arithmetic midpoint of consecutive nodes."""

    a: np.ndarray
    green: np.ndarray   # 3/2 Om / a_j (Poisson prefactor, Phi_k = -green delta_k / k^2)
    c1: np.ndarray
    c2: np.ndarray
    kick: np.ndarray
    drift: np.ndarray
    dD1: np.ndarray
    dD2: np.ndarray
    D1: np.ndarray
    D2: np.ndarray
    dD1da: np.ndarray
    dD2da: np.ndarray


def step_table(c: Cosmology, a_nodes, growth: Growth | None = None, modified: bool = False,
               n_lpt: float = N_LPT) -> StepTable:
    """modified: the Tassev et al. (2013) kick and drift factors (kick about
    the node a_j, drift about the midpoint a_{j+1/2} where the kicked momentum
    sits); otherwise the standard ones."""
    a_nodes = np.asarray(a_nodes, dtype=np.float64)
    n = a_nodes.size
    g = growth if growth is not None else Growth(c)
    D1, dD1da, D2, dD2da = g(a_nodes)
    green = 1.5 * c.omega_m / a_nodes
    kick = np.zeros(n)
    drift = np.zeros(n)
    dD1 = np.zeros(n)
    dD2 = np.zeros(n)
    for j in range(n):
        aj = a_nodes[j]
        if j > 0:
            am = 0.5 * (a_nodes[j - 1] + aj)
            kick[j] += kick_modified(am, aj, aj, c, n_lpt) if modified else kick_integral(am, aj, c)
        if j < n - 1:
            ap = 0.5 * (aj + a_nodes[j + 1])
            kick[j] += kick_modified(aj, ap, aj, c, n_lpt) if modified else kick_integral(aj, ap, c)
            drift[j] = (drift_modified(aj, a_nodes[j + 1], ap, c, n_lpt) if modified
                        else drift_integral(aj, a_nodes[j + 1], c))
            dD1[j] = D1[j + 1] - D1[j]
            dD2[j] = D2[j + 1] - D2[j]
    return StepTable(a=a_nodes, green=green, c1=green * D1, c2=green * (D2 - D1**2),
                     kick=kick, drift=drift, dD1=dD1, dD2=dD2, D1=D1, D2=D2,
                     dD1da=dD1da, dD2da=dD2da)


def lpt_momentum_coeffs(a: float, c: Cosmology, growth: Growth | None = None):
    """p_LPT = a^2 dx_LPT/dt = a^3 E(a) [D1'(a) Psi1 + D2'(a) Psi2]; returns the
    two coefficients multiplying Psi1 and Psi2."""
    g = growth if growth is not None else Growth(c)
    _, dD1, _, dD2 = g(np.array([a]))
    pref = a**3 * float(E(a, c))
    return pref * float(dD1[0]), pref * float(dD2[0])
