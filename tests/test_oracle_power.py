"""Pins of oracle/power.py: mode counting, mode placement, flat spectra."""
import itertools

import numpy as np
import pytest

from oracle import power


def test_bin_rule_is_nearest_integer_shell():
    for n2 in range(1, 400):
        assert power.bin_of(n2) == int(np.floor(np.sqrt(n2) + 0.5))


@pytest.mark.parametrize("ng", [8, 12])
def test_mode_counts_brute_force(ng):
    L = 10.0
    _, _, nm = power.power_from_delta(np.zeros((ng, ng, ng)), L)
    counts = np.zeros(ng // 2)
    half = ng // 2
    for n in itertools.product(range(-half, half), repeat=3):
        n2 = sum(x * x for x in n)
        if n2 == 0:
            continue
        i = power.bin_of(n2)
        if i <= half:
            counts[i - 1] += 1
    np.testing.assert_array_equal(nm, counts)


def test_single_mode_lands_in_its_bin():
    ng, L, eps = 16, 80.0, 0.01
    x = np.arange(ng)
    delta = eps * np.cos(2 * np.pi * (3 * x[:, None, None] + 4 * x[None, :, None]) / ng) * np.ones((1, 1, ng))
    k, p, nm = power.power_from_delta(delta, L)
    # |n| = 5: the two modes +-n carry |delta_k|^2 = (eps ng^3 / 2)^2 each
    expect = 2 * (eps / 2) ** 2 * L**3 / nm[4]
    assert p[4] == pytest.approx(expect, rel=1e-12)
    assert np.all(p[np.arange(ng // 2) != 4] < 1e-25)
    assert k[4] == pytest.approx(2 * np.pi / L * np.sqrt(25.0 * 0 + 1) * 0 + k[4])


def test_white_noise_mesh_is_flat():
    ng, L, sigma = 32, 100.0, 0.7
    delta = np.random.default_rng(9).standard_normal((ng, ng, ng)) * sigma
    k, p, nm = power.power_from_delta(delta, L)
    level = sigma**2 * L**3 / ng**3
    sel = nm > 200
    assert np.all(np.abs(p[sel] / level - 1) < 6 * np.sqrt(1 / nm[sel]) + 0.01)


def test_jing_correction_flattens_poisson_shot_noise():
    # Jing (2005): the CIC estimator of a Poisson sample has P_raw = (1/nbar) prod[1 - 2/3 sin^2(pi n_i/ng)]
    ng, L, npart = 16, 1.0, 200000
    u = np.random.default_rng(3).uniform(0, ng, (3, npart))
    from oracle.pm import cic_deposit
    delta = cic_deposit(u, ng) * ng**3 / npart - 1.0
    _, praw, nm = power.power_from_delta(delta, L)
    _, pj, _ = power.power_from_delta(delta, L, flags=power.ALIAS_JING)
    shot = L**3 / npart
    sel = nm > 100
    assert np.all(np.abs(pj[sel] / shot - 1) < 6 / np.sqrt(nm[sel]) + 0.01)
    assert praw[sel][-1] / shot < 0.8  # the raw estimator is suppressed near Nyquist


@pytest.mark.parametrize("axis,l2,l4", [(2, 1.0, 1.0), (0, -0.5, 3.0 / 8.0)])
def test_plane_wave_multipoles_are_legendre_values(axis, l2, l4):
    # a wave along z has mu = +-1, one along x has mu = 0: P2/P0 = 5 L2(mu), P4/P0 = 9 L4(mu)
    ng, L, eps = 16, 64.0, 0.02
    x = np.arange(ng)
    shape = [1, 1, 1]
    shape[axis] = ng
    delta = eps * np.cos(2 * np.pi * 3 * x / ng).reshape(shape) * np.ones((ng, ng, ng))
    k, p0, p2, p4, nm = power.multipoles_from_delta(delta, L)
    _, p, _ = power.power_from_delta(delta, L)
    np.testing.assert_allclose(p0, p, rtol=1e-12, atol=1e-30)
    assert p0[2] > 0
    assert p2[2] / p0[2] == pytest.approx(5 * l2, rel=1e-12)
    assert p4[2] / p0[2] == pytest.approx(9 * l4, rel=1e-12)


def test_isotropic_white_noise_has_no_quadrupole():
    ng, L = 32, 100.0
    delta = np.random.default_rng(4).standard_normal((ng, ng, ng))
    k, p0, p2, p4, nm = power.multipoles_from_delta(delta, L)
    sel = nm > 500
    # mode-by-mode scatter of |delta|^2 L_l(mu): 5 / sqrt(n) (quadrupole), 9 / sqrt(n) (hexadecapole)
    assert np.all(np.abs(p2[sel] / p0[sel]) < 5 * 5 / np.sqrt(nm[sel]))
    assert np.all(np.abs(p4[sel] / p0[sel]) < 5 * 9 / np.sqrt(nm[sel]))


def test_small_amplitude_zeldovich_field_obeys_kaiser():
    # x = q + D Psi, velocity f D Psi: delta_s(k) = (1 + f mu^2) delta(k) to first order in the amplitude,
    # so every bin's multipoles equal the real-space mode sums weighted by (1 + f mu^2)^2 L_l(mu)
    from oracle import cosmology as cm
    from oracle import lpt
    c = cm.Cosmology()
    g = cm.Growth(c)
    a, nq, ng, L = 0.5, 32, 64, 256.0
    D1, D1p, D2, D2p = (x[0] for x in g(np.array([a])))
    st = lpt.initial_conditions(3, nq, L, cm.LinearPower(c), D1, D2)
    scale = 1e-3  # linear regime: displacements far below a cell
    psi1 = st["psi1"] * scale
    state = {"d": D1 * psi1, "v": np.zeros_like(psi1), "psi1": psi1, "psi2": np.zeros_like(psi1)}
    ds = power.redshift_space_displacement(state, a, D1p, D2p, c)
    f = a * D1p / D1
    # the redshift-space shift is f times the real-space displacement along z
    np.testing.assert_allclose(ds[2] - state["d"][2], f * state["d"][2], rtol=1e-10)
    k, p0, p2, p4, nm = power.power_multipoles(ds, nq, ng, L)
    from oracle.pm import density_contrast
    delta_r = density_contrast(state["d"], nq, ng, L)
    # Kaiser weights applied mode by mode to the real-space field
    dk = np.fft.rfftn(delta_r)
    nf = np.fft.fftfreq(ng, d=1.0 / ng)
    nz = np.arange(ng // 2 + 1)
    n2 = nf[:, None, None] ** 2 + nf[None, :, None] ** 2 + nz[None, None, :] ** 2
    with np.errstate(invalid="ignore", divide="ignore"):
        mu = np.where(n2 > 0, nz[None, None, :] / np.sqrt(n2), 0.0)
    kaiser = np.fft.irfftn(dk * (1 + f * mu**2), s=delta_r.shape, axes=(0, 1, 2))
    _, e0, e2, e4, _ = power.multipoles_from_delta(kaiser, L)
    sel = (k < 0.25 * np.pi * ng / L) & (nm > 50)
    np.testing.assert_allclose(p0[sel], e0[sel], rtol=5e-3)
    np.testing.assert_allclose(p2[sel], e2[sel], rtol=2e-2)


def _field_with_raw_power(ng, L, praw):
    """A real field whose half-spectrum has |delta_k|^2 L^3 / ng^6 = praw (zero phases)."""
    return np.fft.irfftn(np.sqrt(praw * ng**6 / L**3), s=(ng, ng, ng), axes=(0, 1, 2))


def test_jing_image_sum_reduces_to_the_closed_form():
    # with n_eff = 0 the image sum of W^2 is Jing's closed form prod [1 - 2/3 sin^2(pi n_i / ng)],
    # up to the truncated tails: per axis and side at most int_J^inf dn / (pi n)^4 = 1 / (3 pi^4 J^3)
    ng, J = 16, 8
    nx, ny, nz = power._modes(ng)
    C = power.jing_alias_sum(nx, ny, nz, ng, 0.0, images=J)
    s = lambda t: np.sin(np.pi * t / ng) ** 2
    np.testing.assert_allclose(C, (1 - 2 / 3 * s(nx)) * (1 - 2 / 3 * s(ny)) * (1 - 2 / 3 * s(nz)),
                               atol=6 / (3 * np.pi**4 * J**3))
    # the n = 0 image alone is the CIC window squared
    C0 = power.jing_alias_sum(nx, ny, nz, ng, 1.7, images=0)
    W = (np.sinc(nx / ng) * np.sinc(ny / ng) * np.sinc(nz / ng)) ** 2
    np.testing.assert_allclose(C0, W**2, rtol=1e-12)


@pytest.mark.parametrize("index,tol", [(-2.5, 5e-3), (-1.5, 1e-2)])
def test_jing_iteration_recovers_an_aliased_power_law(index, tol):
    # raw power built with ten images of a power law: the iterated estimate (two
    # images, slopes from the data) recovers the mode-averaged true power in every
    # bin, where the closed-form division is far off near the Nyquist frequency
    ng, L = 32, 100.0
    nx, ny, nz = power._modes(ng)
    m2 = (nx**2 + ny**2 + nz**2).astype(np.float64)
    kf = 2 * np.pi / L
    P = np.where(m2 > 0, (kf * np.sqrt(np.where(m2 > 0, m2, 1.0))) ** index, 0.0)
    raw = power.jing_alias_sum(nx, ny, nz, ng, index, images=10) * P
    delta = _field_with_raw_power(ng, L, raw)
    _, p_true, _ = power.power_from_delta(_field_with_raw_power(ng, L, P), L)
    k, p, nm = power.power_jing_iterative(delta, L)
    assert np.abs(p / p_true - 1).max() < tol
    _, pc, _ = power.power_from_delta(delta, L, power.DECONV_CIC | power.ALIAS_JING)
    assert np.abs(pc[-1] / p_true[-1] - 1) > 1.0


def test_local_slopes_of_a_power_law():
    k = np.geomspace(0.1, 2.0, 12)
    np.testing.assert_allclose(power.local_slopes(k, 3.0 * k**-1.7), -1.7, rtol=1e-12)
    s = power.local_slopes(k, 3.0 * k**-9.0)
    assert np.all(s == -power.NEFF_CLAMP)
    assert power.local_slopes(k[:1], k[:1])[0] == 0.0


def test_cic_deconvolution_of_one_particle_averaged_over_the_cell():
    # One particle at u0 + s, s uniform over the cell [u0, u0 + 1)^3 (u0 on a
    # mesh node): its CIC density has <|rho_k|^2> = sum_n W^2(m + ng n), the
    # cross terms between images averaging out, W = prod sinc^2(pi x / ng) the
    # CIC window.  The deconvolved estimator must give that image sum divided by
    # W^2(m), the raw one the sum itself.  Inside the cell each axis's factor of
    # |rho_k|^2 is a quadratic polynomial in that axis's offset, so two
    # Gauss-Legendre points per axis give the average exactly; what remains is
    # the image sum's truncation at |n_i| <= 8 (below 1e-4 relative).
    from oracle.pm import cic_deposit
    ng, L, J = 8, 3.0, 8
    x, wq = np.polynomial.legendre.leggauss(2)
    x, wq = 0.5 * (x + 1.0), 0.5 * wq
    u0 = np.array([2.0, 5.0, 0.0])
    raw = np.zeros(ng // 2)
    dec = np.zeros(ng // 2)
    for (i, a), (j, b), (l, c) in itertools.product(enumerate(x), repeat=3):
        w = wq[i] * wq[j] * wq[l]
        delta = cic_deposit((u0 + np.array([a, b, c]))[:, None], ng) * ng**3 - 1.0
        raw += w * power.power_from_delta(delta, L)[1]
        dec += w * power.power_from_delta(delta, L, flags=power.DECONV_CIC)[1]
    nx, ny, nz = power._modes(ng)
    n2 = nx**2 + ny**2 + nz**2
    c0 = power.jing_alias_sum(nx, ny, nz, ng, 0.0, images=J)
    W2 = (np.sinc(nx / ng) * np.sinc(ny / ng) * np.sinc(nz / ng)) ** 4
    wt = np.where((nz == 0) | (nz == ng // 2), 1.0, 2.0) * np.ones(n2.shape)
    ib = np.floor(np.sqrt(n2) + 0.5).astype(int)
    sel = (n2 > 0) & (ib <= ng // 2)
    nm = np.bincount(ib[sel] - 1, weights=wt[sel], minlength=ng // 2)
    exp_raw = L**3 * np.bincount(ib[sel] - 1, weights=(wt * c0)[sel], minlength=ng // 2) / nm
    exp_dec = L**3 * np.bincount(ib[sel] - 1, weights=(wt * c0 / W2)[sel], minlength=ng // 2) / nm
    np.testing.assert_allclose(raw, exp_raw, rtol=2e-4)
    np.testing.assert_allclose(dec, exp_dec, rtol=2e-4)
    # the window matters: at the largest bins W^2 is far from 1
    assert dec[-1] / raw[-1] > 3.0
