"""Pins of oracle/cola.py: Zel'dovich exactness and linear growth."""
import numpy as np
import pytest

from oracle import cola, lpt, power
from oracle import cosmology as cm
from synth import plane_wave_psi1


def _zeldovich_error(nq, m, kA, L=64.0):
    c = cm.Cosmology()
    g = cm.Growth(c)
    tab = cm.step_table(c, cm.time_nodes(0.05, 1.0, 40), g)
    psi1 = plane_wave_psi1(nq, L, kA)  # delta = kA cos(k q), shell crossing at kA D1 = 1
    st = {"psi1": psi1, "psi2": np.zeros_like(psi1), "d": tab.D1[0] * psi1, "v": np.zeros_like(psi1)}
    cola.run(st, tab, nq, nq * m, L)
    ref = tab.D1[-1] * psi1
    p_lpt = cm.lpt_momentum_coeffs(1.0, c, g)[0] * psi1
    return (np.linalg.norm(st["d"] - ref) / np.linalg.norm(ref),
            np.linalg.norm(st["v"]) / np.linalg.norm(p_lpt))


@pytest.mark.slow
def test_zeldovich_plane_wave_is_exact_before_shell_crossing():
    # 1D: the Zel'dovich trajectory is the exact solution, so the COLA residual
    # stays ~0 and only the mesh error remains, shrinking with resolution.
    e32, v32 = _zeldovich_error(32, 3, 0.5)
    e16, _ = _zeldovich_error(16, 3, 0.5)
    assert e32 < 1.5e-2
    assert v32 < 1e-2
    assert e32 < 0.5 * e16


def _linear_growth_ratio(nq):
    c = cm.Cosmology(sigma8=1e-3)
    g = cm.Growth(c)
    P = cm.LinearPower(c)
    L = 4.0 * nq
    tab = cm.step_table(c, cm.time_nodes(0.05, 1.0, 40), g)
    st = lpt.initial_conditions(1, nq, L, P, tab.D1[0], tab.D2[0])
    _, p0, _ = power.power_spectrum(st["d"], nq, 2 * nq, L)
    cola.run(st, tab, nq, 3 * nq, L)
    _, p1, _ = power.power_spectrum(st["d"], nq, 2 * nq, L)
    return p1 / p0 / (tab.D1[-1] / tab.D1[0]) ** 2


@pytest.mark.slow
def test_linear_regime_power_grows_as_D1_squared():
    r32 = _linear_growth_ratio(32)
    r16 = _linear_growth_ratio(16)
    # large scales follow linear theory; the lattice/mesh deficit is O((k dq)^2)
    assert abs(r32[0] - 1) < 0.012
    assert abs(r32[1] - 1) < 0.04
    assert 3.0 < (1 - r16[0]) / (1 - r32[0]) < 5.5
