"""COLA time stepping in the frame comoving with the 2LPT trajectories
(Eq. 1: x_res = x - x_LPT; Eq. 2: d^2 x_res/dt^2 = -grad Phi - d^2 x_LPT/dt^2,
with only the left-hand side discretised).

Test infrastructure only (see ``oracle/__init__``).

Reading (the paper gives no discretisation): kick-drift-kick leapfrog on the
nodes of Eq. 3 with the standard factors K and Dr of ``cosmology.step_table``.
The state is the total displacement d = x - q and the residual momentum
v = p - p_LPT (p = a^2 dx/dt).  The LPT acceleration follows from the growth
equations:  d/dt(a^2 d/dt [D1 Psi1 + D2 Psi2]) = 3/2 Om/a [D1 Psi1 + (D2-D1^2) Psi2].
Node j: A_j = F(x_j) - c1_j Psi1 - c2_j Psi2; v += kick_j A_j; then, except at
the last node, d += drift_j v + dD1_j Psi1 + dD2_j Psi2.
The PM-only variant (App. B) uses the same loop with the LPT frame removed
(c1 = c2 = dD1 = dD2 = 0 after the initial displacement, v started at p_LPT).

Pins (tests/test_oracle_cola.py): a 1D plane wave before shell crossing, for
which the 1LPT trajectory is the exact solution, keeps v ~ 0 and d ~ D1 Psi1;
in the linear regime P(k) grows as D1(a)^2.
"""
from __future__ import annotations

import numpy as np

from .cosmology import StepTable
from .pm import pm_force


def cola_step(state: dict, j: int, tab: StepTable, nq: int, ng: int, L: float, pm_only=False):
    """Advance the state (in place) through node j: force, kick, drift."""
    n = tab.a.size
    d, v, psi1, psi2 = state["d"], state["v"], state["psi1"], state["psi2"]
    F = pm_force(d, nq, ng, L, tab.green[j])
    if pm_only:
        A = F
    else:
        A = F - tab.c1[j] * psi1 - tab.c2[j] * psi2
    v += tab.kick[j] * A
    if j < n - 1:
        if pm_only:
            d += tab.drift[j] * v
        else:
            d += tab.drift[j] * v + tab.dD1[j] * psi1 + tab.dD2[j] * psi2
    return state


def run(state: dict, tab: StepTable, nq: int, ng: int, L: float, steps=None, pm_only=False):
    n = tab.a.size
    for j in range(n) if steps is None else steps:
        cola_step(state, j, tab, nq, ng, L, pm_only=pm_only)
    return state


def snapshot_displacement(state: dict, a_node: float, a_out: float, growth, c, tab_drift):
    """Displacement at a_out from a state whose positions sit at node a_node and
    whose momentum is the one used for the drift that reached a_node:
    d_out = d + Dr(a_node, a_out) v + [D1(a_out)-D1(a_node)] Psi1 + [D2(a_out)-D2(a_node)] Psi2.
    No extra force evaluation; the trajectory itself is untouched."""
    D1, _, D2, _ = growth(np.array([a_node, a_out]))
    dr = tab_drift(a_node, a_out, c)
    return (state["d"] + dr * state["v"] + (D1[1] - D1[0]) * state["psi1"]
            + (D2[1] - D2[0]) * state["psi2"])
