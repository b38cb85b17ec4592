"""Pins of oracle/pm.py and oracle/dft.py."""
import math

import numpy as np
import pytest
from scipy.special import erfc

from oracle import dft, pm
from synth import random_displacements, single_mode_delta


@pytest.mark.parametrize("shape", [(6, 6, 6), (8, 8, 8), (10, 10, 10), (12, 12, 12), (6, 10, 12), (30, 6, 10)])
def test_numpy_fft_matches_direct_dft(shape):
    x = np.random.default_rng(1).standard_normal(shape)
    ref = dft.rdftn(x)
    got = np.fft.rfftn(x)
    assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()
    back = np.real(dft.dftn(dft.dftn(x), +1)) / x.size
    np.testing.assert_allclose(back, x, atol=1e-12)
    import scipy.fft  # the threaded backend of oracle.lpt for full-size references
    assert np.abs(scipy.fft.rfftn(x, workers=2) - ref).max() <= 1e-12 * np.abs(ref).max()


def test_direct_dft_single_mode():
    n = 12
    x = np.cos(2 * np.pi * 3 * np.arange(n) / n)
    X = dft.dftn(x)
    expect = np.zeros(n, complex)
    expect[3] = expect[n - 3] = n / 2
    np.testing.assert_allclose(X, expect, atol=1e-12)


def test_cic_sum_equals_particle_count():
    nq, ng, L = 8, 24, 50.0
    d = random_displacements(3, nq, 7.0).astype(np.float64)
    rho = pm.cic_deposit(pm.mesh_coords(d, nq, ng, L), ng)
    assert rho.sum() == pytest.approx(nq**3, rel=1e-13)
    assert rho.min() >= 0
    delta = pm.density_contrast(d, nq, ng, L)
    assert abs(delta.mean()) < 1e-13


def test_particle_on_node_fills_one_cell():
    ng = 10
    u = np.array([[3.0], [9.0], [0.0]])
    rho = pm.cic_deposit(u, ng)
    assert rho[3, 9, 0] == 1.0 and np.count_nonzero(rho) == 1
    # periodic wrap: a particle just below ng shares with cell 0
    u = np.array([[9.5], [0.0], [0.0]])
    rho = pm.cic_deposit(u, ng)
    assert rho[9, 0, 0] == 0.5 and rho[0, 0, 0] == 0.5


def test_unperturbed_lattice_sits_at_cell_midpoints():
    nq, ng, L = 4, 12, 12.0
    u = pm.mesh_coords(np.zeros((3, nq**3)), nq, ng, L)
    assert np.allclose(u - np.floor(u), 0.5)
    delta = pm.density_contrast(np.zeros((3, nq**3)), nq, ng, L)
    F = pm.force_mesh_from_delta(delta, L, 1.0)
    Fp = np.stack([pm.cic_gather(F[j], u) for j in range(3)])
    assert np.abs(Fp).max() < 1e-12  # a perfect lattice feels no force


def test_deposit_gather_adjoint():
    # sum_c rho(c) f(c) = sum_p (gather f)(p): the same CIC weights both ways
    ng, n = 16, 500
    rng = np.random.default_rng(5)
    u = rng.uniform(0, ng, (3, n))
    f = rng.standard_normal((ng, ng, ng))
    lhs = (pm.cic_deposit(u, ng) * f).sum()
    rhs = pm.cic_gather(f, u).sum()
    assert lhs == pytest.approx(rhs, rel=1e-12)
    # partition of unity: a constant field is gathered exactly
    assert np.allclose(pm.cic_gather(np.full((ng, ng, ng), 2.5), u), 2.5)


def test_single_fourier_mode_closed_form():
    ng, L, eps, green = 24, 100.0, 0.3, 0.7
    for nvec in [(1, 0, 0), (2, 3, 0), (1, -2, 5), (0, 0, 11)]:
        delta = single_mode_delta(ng, L, eps, nvec)
        F = pm.force_mesh_from_delta(delta, L, green)
        k = 2 * np.pi * np.asarray(nvec, float) / L
        x = np.arange(ng) * L / ng
        phase = k[0] * x[:, None, None] + k[1] * x[None, :, None] + k[2] * x[None, None, :]
        k2 = (k**2).sum()
        for j in range(3):
            expect = -green * eps * k[j] / k2 * np.sin(phase)
            assert np.abs(F[j] - expect).max() < 1e-12 * max(1.0, np.abs(expect).max())


def test_nyquist_gradient_is_zero():
    ng, L = 8, 8.0
    delta = single_mode_delta(ng, L, 1.0, (4, 1, 0))  # n_x at Nyquist
    F = pm.force_mesh_from_delta(delta, L, 1.0)
    assert np.abs(F[0]).max() < 1e-12
    assert np.abs(F[1]).max() > 0.01


def test_net_force_vanishes():
    nq, ng, L = 8, 24, 64.0
    d = random_displacements(11, nq, 10.0).astype(np.float64)
    F = pm.pm_force(d, nq, ng, L, 1.5)
    assert np.abs(F.sum(axis=1)).max() <= 1e-12 * np.abs(F).sum()


def _ewald_grad(r, L, alpha, nreal=2, nk=7):
    """Gradient of the periodic Green's function G (lap G = delta_D - 1/L^3) by
    Ewald summation (real-space erfc images + reciprocal-space Gaussian sum)."""
    g = np.zeros_like(r)
    for a in range(-nreal, nreal + 1):
        for b in range(-nreal, nreal + 1):
            for c in range(-nreal, nreal + 1):
                s = r + np.array([a, b, c]) * L
                d = np.linalg.norm(s, axis=-1)[..., None]
                g += s / d * (erfc(alpha * d) / d**2 + 2 * alpha / math.sqrt(math.pi) * np.exp(-(alpha * d) ** 2) / d) / (4 * math.pi)
    kf = 2 * math.pi / L
    n = np.arange(-nk, nk + 1)
    kv = np.stack(np.meshgrid(n, n, n, indexing="ij"), -1).reshape(-1, 3) * kf
    kv = kv[np.any(kv != 0, axis=1)]
    k2 = (kv**2).sum(1)
    coef = kv / k2[:, None] * np.exp(-k2 / (4 * alpha**2))[:, None] / L**3
    g += np.sin(r @ kv.T) @ coef
    return g


def test_single_particle_matches_ewald_inverse_square():
    # one unit-count particle on an ng^3 mesh: delta = rho ng^3 - 1, so
    # lap Phi = green (L^3 delta_D - 1) and F = -green L^3 grad G.
    ng, L, green = 32, 32.0, 1.0
    rng = np.random.default_rng(2)
    ratios, tang = [], []
    for _ in range(6):
        x0 = rng.uniform(0, ng, 3)
        delta = pm.cic_deposit(x0[:, None], ng) * ng**3 - 1.0
        fm = pm.force_mesh_from_delta(delta, L, green)
        dirs = rng.standard_normal((400, 3))
        dirs /= np.linalg.norm(dirs, axis=1)[:, None]
        r = rng.uniform(4.0, 8.0, 400)  # 4 cells .. ng/4
        sep = dirs * r[:, None]
        pts = np.mod(x0 + sep, ng)
        F = np.stack([pm.cic_gather(fm[j], pts.T) for j in range(3)], 1)
        Fe = -green * L**3 * _ewald_grad(sep * (L / ng), L, alpha=5.0 / L)
        rad = (F * dirs).sum(1)
        rad_e = (Fe * dirs).sum(1)
        assert np.all(rad_e < 0)  # attractive
        ratios.append(rad / rad_e)
        tang.append(np.linalg.norm(F - rad[:, None] * dirs, axis=1) / np.abs(rad_e))
    ratios = np.concatenate(ratios)
    # the ik gradient rings at the cell scale, but on average the PM force is 1/r^2
    assert abs(ratios.mean() - 1.0) < 0.02
    assert np.median(np.abs(ratios - 1.0)) < 0.06
    assert np.concatenate(tang).mean() < 0.1
    # the Ewald sum itself: point-mass limit 1/(4 pi r^2) close to the source
    r_small = 0.02 * L
    g_small = _ewald_grad(np.array([[r_small, 0.0, 0.0]]), L, alpha=5.0 / L)[0, 0]
    assert g_small == pytest.approx(1.0 / (4 * math.pi * r_small**2), rel=2e-3)
    # and by symmetry no force half a box away
    assert np.abs(_ewald_grad(np.array([[L / 2, 0.0, 0.0]]), L, alpha=5.0 / L)).max() < 1e-12


def test_radial_filter_constant_and_hat_nodes():
    # T = const is that constant everywhere (also past the last node); the hat
    # on node b is 1 at k_b = b kmax / (nb - 1), 0 at the neighbouring nodes
    # and 1/2 half-way: the node spacing and the interpolation
    nb, kmax = 9, 4.0
    k = np.linspace(0.0, 1.3 * kmax, 1001)
    np.testing.assert_allclose(pm.radial_filter(k, np.full(nb, 0.625), kmax), 0.625, rtol=0, atol=1e-15)
    dk = kmax / (nb - 1)
    for b in (0, 3, nb - 1):
        T = np.zeros(nb)
        T[b] = 1.0
        at = lambda kk: float(pm.radial_filter(np.array([kk]), T, kmax)[0])
        assert at(b * dk) == pytest.approx(1.0, abs=1e-15)
        for nbr in (b - 1, b + 1):
            if 0 <= nbr < nb:
                assert at(nbr * dk) == pytest.approx(0.0, abs=1e-15)
                assert at(0.5 * (b + nbr) * dk) == pytest.approx(0.5, abs=1e-15)


def test_filtered_force_mesh_node_spacing():
    # inside force_mesh_from_delta the nodes sit at b sqrt(3) pi ng / (L (nb - 1)).
    # A diagonal mode n = (m, m, m) has |k| = 2 pi sqrt(3) m / L, which is node b
    # exactly when m = ng b / (2 (nb - 1)): ng = 16, nb = 9, b = 4 gives m = 4.
    # The hat on node 4 passes that mode whole, the hats on nodes 3 and 5 not at
    # all; a constant filter scales the force.
    ng, L, eps, green = 16, 40.0, 0.2, 0.9
    delta = single_mode_delta(ng, L, eps, (4, 4, 4))
    F = pm.force_mesh_from_delta(delta, L, green)
    tol = 1e-12 * np.abs(F).max()
    np.testing.assert_allclose(pm.force_mesh_from_delta(delta, L, green, filt=np.full(5, 1.75)), 1.75 * F,
                               rtol=0, atol=tol)
    for b, expect in ((4, 1.0), (3, 0.0), (5, 0.0)):
        T = np.zeros(9)
        T[b] = 1.0
        np.testing.assert_allclose(pm.force_mesh_from_delta(delta, L, green, filt=T), expect * F, rtol=0, atol=tol)


@pytest.mark.parametrize("m", [1, 2, 3, 4])
@pytest.mark.parametrize("axis", [0, 1, 2])
def test_lattice_wave_force_equals_the_full_mesh_force(m, axis):
    # the reduced periodic cell against brute force: pm_force on the whole mesh
    nq, L, green = 8, 24.0, 0.8
    ng = nq * m
    dline = np.random.default_rng(10 * m + axis).standard_normal(nq) * 0.6 * L / nq
    d = np.zeros((3, nq**3))
    d[axis] = dline[pm.lagrangian_index(nq)[axis]]
    full = pm.pm_force(d, nq, ng, L, green)
    red = pm.lattice_wave_force(dline, nq, ng, L, green, axis)
    assert np.abs(red - full).max() <= 1e-12 * np.abs(full).max()
    assert np.abs(full[axis]).max() > 0.05
