"""Pins of oracle/cosmology.py against closed forms and textbook limits."""
import math
import os

import numpy as np
import pytest

from oracle import cosmology as cm

HERE = os.path.dirname(__file__)
EDS = cm.Cosmology(omega_m=1.0, omega_l=0.0)
LCDM = cm.Cosmology()


def test_eds_growth_closed_forms():
    # Einstein-de Sitter: D1 = a, D2 = -3/7 a^2 exactly (normalised D1(1)=1)
    a = np.array([0.01, 0.05, 0.3, 0.77, 1.0])
    D1, dD1, D2, dD2 = cm.Growth(EDS)(a)
    np.testing.assert_allclose(D1, a, rtol=1e-11)
    np.testing.assert_allclose(dD1, 1.0, rtol=1e-11)
    np.testing.assert_allclose(D2, -3.0 / 7.0 * a**2, rtol=1e-10)
    np.testing.assert_allclose(dD2, -6.0 / 7.0 * a, rtol=1e-10)


def test_eds_kick_drift_closed_forms():
    # E = a^-3/2: K = int da a^1/2 = 2/3 (b^3/2 - a^3/2); Dr = int da a^-3/2 = -2 (b^-1/2 - a^-1/2)
    for a, b in [(0.05, 0.074359), (0.3, 0.31), (0.9, 1.0)]:
        assert cm.kick_integral(a, b, EDS) == pytest.approx(2.0 / 3.0 * (b**1.5 - a**1.5), rel=1e-12)
        assert cm.drift_integral(a, b, EDS) == pytest.approx(-2.0 * (b**-0.5 - a**-0.5), rel=1e-12)


@pytest.mark.parametrize("n", [-2.5, -1.0, 1.5])
def test_eds_modified_kick_drift_closed_forms(n):
    # E = a^-3/2: kick = (b^n - a^n) ac^(3/2 - n) / n; drift = ac^-n (b^(n-1/2) - a^(n-1/2)) / (n - 1/2)
    for a, b in [(0.05, 0.074359), (0.3, 0.31), (0.9, 1.0)]:
        ac = 0.5 * (a + b)
        assert cm.kick_modified(a, b, ac, EDS, n) == pytest.approx((b**n - a**n) * ac ** (1.5 - n) / n, rel=1e-12)
        assert cm.drift_modified(a, b, ac, EDS, n) == pytest.approx(
            ac**-n * (b ** (n - 0.5) - a ** (n - 0.5)) / (n - 0.5), rel=1e-12)


def test_modified_factors_reduce_to_the_standard_ones_on_short_steps():
    # over a step of width h about its midpoint the power-law momentum agrees with
    # a constant force (kick) and a constant momentum (drift) up to O(h^2): the
    # relative difference falls four-fold when h halves
    for a0 in (0.05, 0.3, 0.9):
        rel = []
        for h in (4e-3, 2e-3):
            a, b = a0, a0 + h
            ac = 0.5 * (a + b)
            rel.append((cm.kick_modified(a, b, ac, LCDM) / cm.kick_integral(a, b, LCDM) - 1,
                        cm.drift_modified(a, b, ac, LCDM) / cm.drift_integral(a, b, LCDM) - 1))
        for q in range(2):
            assert abs(rel[0][q]) < 2e-2
            assert rel[0][q] / rel[1][q] == pytest.approx(4.0, rel=0.05), (a0, q, rel)


def test_modified_step_table_uses_the_node_and_the_midpoint():
    # kick about the node where the force is, drift about the midpoint where the kicked momentum is
    a = cm.time_nodes(0.05, 1.0, 6)
    tab = cm.step_table(LCDM, a, modified=True)
    std = cm.step_table(LCDM, a)
    for j in range(6):
        k = 0.0
        if j > 0:
            k += cm.kick_modified(0.5 * (a[j - 1] + a[j]), a[j], a[j], LCDM)
        if j < 5:
            k += cm.kick_modified(a[j], 0.5 * (a[j] + a[j + 1]), a[j], LCDM)
            assert tab.drift[j] == pytest.approx(cm.drift_modified(a[j], a[j + 1], 0.5 * (a[j] + a[j + 1]), LCDM),
                                                 rel=1e-12)
        assert tab.kick[j] == pytest.approx(k, rel=1e-12)
    np.testing.assert_array_equal(tab.dD1, std.dD1)
    assert np.all(tab.kick != std.kick) and np.all(tab.drift[:-1] != std.drift[:-1])


def test_lcdm_d1_heath_vs_ode():
    a = np.array([0.05, 0.1, 0.33, 0.5, 0.8, 1.0])
    D1 = cm.Growth(LCDM)(a)[0]
    np.testing.assert_allclose(D1, cm.D1_heath(a, LCDM), rtol=1e-10)


def test_lcdm_d2_limits():
    g = cm.Growth(LCDM)
    a = np.array([1e-3, 0.05, 0.5, 1.0])
    D1, _, D2, _ = g(a)
    ratio = D2 / (-3.0 / 7.0 * D1**2)
    # early times: matter domination, D2 -> -3/7 D1^2
    assert abs(ratio[0] - 1.0) < 1e-7
    # Bouchet et al. (1995): D2 ~ -3/7 D1^2 Om(a)^(-1/143), good to ~1e-3
    fit = cm.omega_m_of_a(a, LCDM) ** (-1.0 / 143.0)
    np.testing.assert_allclose(ratio, fit, rtol=1.5e-3)


def test_lcdm_growth_rate_wang_steinhardt():
    # f = dlnD1/dlna ~ Om(a)^gamma, gamma = 6/11 + 15/1331 (1 - Om(a)) for w = -1
    # (Wang & Steinhardt 1998, second-order expansion), good to a few 1e-3
    a = np.array([0.1, 0.5, 1.0])
    D1, dD1, _, _ = cm.Growth(LCDM)(a)
    f = dD1 * a / D1
    om = cm.omega_m_of_a(a, LCDM)
    gamma = 6.0 / 11.0 + 15.0 / 1331.0 * (1.0 - om)
    np.testing.assert_allclose(f, om**gamma, rtol=4e-3)


def test_sigma_R_flat_spectrum_closed_form():
    # P = A up to K: sigma_R^2 = A/(2 pi^2 R^3) int_0^{KR} x^2 W(x)^2 dx with
    # int_0^X x^2 W^2 dx = 3 (2X^3 Si(2X) + X^2 (cos 2X - 3) + 2X sin 2X + cos 2X - 1) / (2 X^3),
    # whose X -> inf limit 3 pi / 2 gives the Parseval value 3A / (4 pi R^3).
    from scipy.special import sici
    A = 123.0
    for R, K in ((2.0, 50.0), (8.0, 3.0), (8.0, 200.0)):
        X = K * R
        F = 3 * (2 * X**3 * sici(2 * X)[0] + X**2 * (math.cos(2 * X) - 3) + 2 * X * math.sin(2 * X)
                 + math.cos(2 * X) - 1) / (2 * X**3)
        s = cm.sigma_R(lambda k: np.full_like(np.asarray(k, dtype=float), A), R, kmax=K)
        assert s**2 == pytest.approx(A / (2 * math.pi**2 * R**3) * F, rel=1e-9)
    assert 3 * math.pi / 2 / (2 * math.pi**2) == pytest.approx(3 / (4 * math.pi))


def test_tophat_window_limits():
    x = np.array([0.0, 1e-4, 5e-4, 2e-3, 1.0, 4.4934094579])  # last: first zero of tan x = x
    w = cm.tophat_window(x)
    assert w[0] == 1.0
    np.testing.assert_allclose(w[1:4], 3 * (np.sin(x[1:4]) - x[1:4] * np.cos(x[1:4])) / x[1:4] ** 3, rtol=1e-6)
    assert abs(w[5]) < 1e-9


def test_eh_transfer_limits():
    T = cm.transfer_eh_nowiggle(np.array([1e-7, 1e-5]), LCDM)
    np.testing.assert_allclose(T, 1.0, atol=1e-5)
    # deep small-scale limit: C0 -> 14.2, gamma_eff -> Om h alpha
    k = np.array([1e5])
    c = LCDM
    om_h2 = c.omega_m * c.h**2
    fb = c.omega_b / c.omega_m
    alpha = 1 - 0.328 * math.log(431 * om_h2) * fb + 0.38 * math.log(22.3 * om_h2) * fb**2
    q = k * (c.t_cmb / 2.7) ** 2 / (c.omega_m * c.h * alpha)
    asym = np.log(2 * math.e + 1.8 * q) / (14.2 * q**2)
    np.testing.assert_allclose(cm.transfer_eh_nowiggle(k, c), asym, rtol=1e-3)
    # monotone decreasing (the no-wiggle form has no oscillations)
    kk = np.logspace(-4, 2, 400)
    assert np.all(np.diff(cm.transfer_eh_nowiggle(kk, c)) < 0)


def test_linear_power_sigma8():
    P = cm.LinearPower(LCDM)
    assert cm.sigma_R(P, 8.0) == pytest.approx(0.8, rel=1e-9)
    assert P(np.array([0.0]))[0] == 0.0


def test_paper_time_node_examples():
    # Sec. 4.3 / Eq. 3: starting at a_i equal to the step width
    for line in open(os.path.join(HERE, "golden", "paper_time_nodes.txt")):
        parts = line.split()
        if not parts or parts[0].startswith("#"):
            continue
        if parts[0] == "nodes":
            n, zi = int(parts[1]), float(parts[2])
            a_i = 1.0 / (1.0 + zi)
            nodes = cm.time_nodes(a_i, 1.0, n)
            assert nodes[1] - nodes[0] == pytest.approx(a_i, rel=1e-12)
            assert nodes[-1] == pytest.approx(1.0, rel=1e-15)
            assert len(nodes) == n
        elif parts[0] == "cell":
            npart, L, m, cell = int(parts[1]), float(parts[2]), int(parts[3]), float(parts[4])
            assert L / (npart * m) == pytest.approx(cell, rel=1e-12)


def test_time_node_variants():
    lin = cm.time_nodes(0.05, 1.0, 40)
    assert np.allclose(np.diff(lin), 0.95 / 39)
    lg = cm.time_nodes(0.025, 1.0, 40, "log")
    assert np.allclose(np.diff(np.log(lg)), math.log(40) / 39)
    pw = cm.time_nodes(0.025, 1.0, 40, "pow", 0.8)
    assert np.allclose(np.diff(pw**0.8), (1 - 0.025**0.8) / 39)


def test_step_table_structure():
    c = LCDM
    a = cm.time_nodes(0.05, 1.0, 6)
    t = cm.step_table(c, a)
    # first node: only the half kick forward; last node: only the closing half kick, no drift
    assert t.kick[0] == pytest.approx(cm.kick_integral(a[0], 0.5 * (a[0] + a[1]), c))
    assert t.kick[-1] == pytest.approx(cm.kick_integral(0.5 * (a[-2] + a[-1]), a[-1], c))
    assert t.drift[-1] == 0.0 and t.dD1[-1] == 0.0
    # total kick over the run = K(a_0, a_last)
    assert t.kick.sum() == pytest.approx(cm.kick_integral(a[0], a[-1], c), rel=1e-12)
    assert t.drift[:-1].sum() == pytest.approx(cm.drift_integral(a[0], a[-1], c), rel=1e-12)
    np.testing.assert_allclose(t.green, 1.5 * c.omega_m / a)


def test_lpt_frame_coefficients_satisfy_equation_of_motion():
    # d/dt (a^2 dD/dt) with d/dt = a E d/da must equal c1 (for D1) and c2 (for D2):
    # the LPT acceleration of Eq. 2, checked by numerical differentiation of the growth.
    c = LCDM
    g = cm.Growth(c)
    for a in (0.07, 0.4, 0.9):
        h = 1e-4 * a
        aa = np.array([a - h, a, a + h])
        D1, dD1, D2, dD2 = g(aa)
        mom1 = aa**3 * cm.E(aa, c) * dD1   # a^2 dD/dt = a^3 E dD/da
        mom2 = aa**3 * cm.E(aa, c) * dD2
        acc1 = a * float(cm.E(a, c)) * (mom1[2] - mom1[0]) / (2 * h)
        acc2 = a * float(cm.E(a, c)) * (mom2[2] - mom2[0]) / (2 * h)
        t = cm.step_table(c, np.array([a, a + 0.01]), g)
        assert acc1 == pytest.approx(t.c1[0], rel=1e-6)
        assert acc2 == pytest.approx(t.c2[0], rel=1e-6)


def test_eh_transfer_depends_on_k_only_through_its_shape_variable():
    # without baryons the fit is a function of q = k Theta^2 / (Omega_m h) (k in h/Mpc):
    # two cosmologies agree at k scaled by their Omega_m h, and a CMB temperature enters as Theta^2
    from dataclasses import replace
    k = np.geomspace(1e-3, 30.0, 40)
    a = replace(LCDM, omega_b=0.0, omega_m=0.25, omega_l=0.75, h=0.7)
    b = replace(LCDM, omega_b=0.0, omega_m=0.3, omega_l=0.7, h=0.6)
    np.testing.assert_allclose(cm.transfer_eh_nowiggle(k, a),
                               cm.transfer_eh_nowiggle(k * (0.3 * 0.6) / (0.25 * 0.7), b), rtol=1e-12)
    hot = replace(a, t_cmb=2.7255 * 1.1)
    np.testing.assert_allclose(cm.transfer_eh_nowiggle(k, hot), cm.transfer_eh_nowiggle(k * 1.1**2, a), rtol=1e-12)


def test_eh_baryon_suppression_vanishes_on_large_scales():
    # the baryons' shape suppression switches on at k ~ 1/s (s ~ 150 Mpc): far below it
    # the fit equals the zero-baryon one with the same Omega_m h, far above it it is lower
    from dataclasses import replace
    nob = replace(LCDM, omega_b=0.0)
    k = np.array([1e-3, 3e-3])
    np.testing.assert_allclose(cm.transfer_eh_nowiggle(k, LCDM), cm.transfer_eh_nowiggle(k, nob), rtol=1e-5)
    assert cm.transfer_eh_nowiggle(3e-3, LCDM) < 0.99  # the check above is not just T ~ 1
    assert cm.transfer_eh_nowiggle(1.0, LCDM) < 0.9 * cm.transfer_eh_nowiggle(1.0, nob)


def test_eh_transfer_matches_the_hand_worked_example():
    # tests/golden/eh98_nowiggle_worked_example.txt: Eqs. 26 and 28-31 of
    # Eisenstein & Hu (1998) worked one at a time for the Sec. 2.1 cosmology;
    # a wrong digit in any of the fit's constants moves T0 at one of the three k
    rows = [line.split()[1:] for line in open(os.path.join(HERE, "golden", "eh98_nowiggle_worked_example.txt"))
            if line.startswith("k_T0")]
    k = np.array([float(r[0]) for r in rows])
    t0 = np.array([float(r[1]) for r in rows])
    assert len(rows) == 3
    np.testing.assert_allclose(cm.transfer_eh_nowiggle(k, LCDM), t0, rtol=2e-8)
