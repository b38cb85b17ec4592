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
