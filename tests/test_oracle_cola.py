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


@pytest.mark.parametrize("j", [0, 17, 38])
def test_snapshot_to_the_next_node_is_the_step_drift(j):
    # A snapshot taken at a_out = a_{j+1} from node j's state after its kick
    # (positions still at a_j) is exactly the drift that the step itself makes:
    # same interval, same signs, same growth differences.
    c = cm.Cosmology()
    g = cm.Growth(c)
    tab = cm.step_table(c, cm.time_nodes(0.05, 1.0, 40), g)
    nq, ng, L = 8, 16, 32.0
    rng = np.random.default_rng(5 + j)
    st = {k: rng.standard_normal((3, nq**3)) * s for k, s in (("d", 0.4), ("v", 2.0), ("psi1", 1.0), ("psi2", 0.3))}
    d0 = st["d"].copy()
    cola.cola_step(st, j, tab, nq, ng, L)
    kicked = dict(st, d=d0)
    snap = cola.snapshot_displacement(kicked, tab.a[j], tab.a[j + 1], g, c, cm.drift_integral)
    np.testing.assert_allclose(snap, st["d"], rtol=0, atol=1e-13 * np.abs(st["d"]).max())
    # and a snapshot at the node itself moves nothing
    same = cola.snapshot_displacement(kicked, tab.a[j], tab.a[j], g, c, cm.drift_integral)
    np.testing.assert_array_equal(same, d0)
