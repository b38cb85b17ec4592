"""Pins of oracle/fof.py: friends-of-friends groups, Warren masses, mass function."""
import itertools
import os

import numpy as np
import pytest

from oracle import fof


def _clumpy(seed, nq, L, nclump=6, spread=0.25):
    """Displacements that pull the lattice into a few tight clumps (spacing units x L/nq)."""
    rng = np.random.default_rng(seed)
    q = fof.lattice_sites(nq).astype(np.float64)
    centres = rng.uniform(0, nq, (nclump, 3))
    which = rng.integers(0, nclump + 2, nq**3)  # two extra labels: stay near the lattice site
    target = q.copy()
    clumped = which < nclump
    target[:, clumped] = centres[which[clumped]].T + rng.normal(0, spread, (3, clumped.sum()))
    target[:, ~clumped] += rng.normal(0, 0.05, (3, (~clumped).sum()))
    return ((target - q) * (L / nq)).astype(np.float32)


def _brute_force(d, nq, L, b):
    """O(N^2) groups from FP64 minimum-image distances and a plain union-find."""
    s = fof.lattice_sites(nq) + d.astype(np.float64) * (nq / L)
    n = s.shape[1]
    parent = list(range(n))

    def find(x):
        while parent[x] != x:
            x = parent[x]
        return x

    gaps = []
    for p in range(n):
        dl = s[:, p + 1:] - s[:, p:p + 1]
        dl -= nq * np.round(dl / nq)
        r = np.sqrt((dl**2).sum(axis=0))
        gaps.append(np.abs(r - b).min() if r.size else np.inf)
        for q in np.nonzero(r <= b)[0] + p + 1:
            a, c = find(p), find(int(q))
            if a != c:
                parent[max(a, c)] = min(a, c)
    return np.array([find(p) for p in range(n)]), min(gaps)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_groups_match_brute_force(seed):
    nq, L, b = 8, 16.0, 0.2
    for s in range(seed, seed + 50, 3):  # inputs with no pair within 1e-4 of b: FP32 and FP64 agree
        d = _clumpy(s, nq, L)
        want, gap = _brute_force(d, nq, L, b)
        if gap > 1e-4:
            break
    else:
        pytest.fail("no input without borderline pairs")
    got = fof.fof_groups(d, nq, L, b)
    np.testing.assert_array_equal(got, want)
    assert len(np.unique(got)) < nq**3 * 0.8  # the clumps do link
    assert (np.bincount(got)[np.unique(got)] > 1).sum() >= 3


def _place(nq, L, targets):
    """Displacements that put particle p at targets[p] (spacing units), others on their sites."""
    q = fof.lattice_sites(nq).astype(np.float64)
    t = q.copy()
    for p, x in targets.items():
        t[:, p] = x
    return ((t - q) * (L / nq)).astype(np.float32)


@pytest.mark.parametrize("step,one_group", [(0.19, True), (0.21, False)])
def test_chain_across_the_periodic_boundary(step, one_group):
    nq, L = 4, 4.0
    chain = [1, 7, 20, 33, 46, 59]
    d = _place(nq, L, {p: ((3.55 + step * m) % nq, 0.5, 0.5) for m, p in enumerate(chain)})
    g = fof.fof_groups(d, nq, L, 0.2)
    if one_group:
        assert np.all(g[chain] == min(chain))
    else:
        assert len(np.unique(g[chain])) == len(chain)
    others = np.setdiff1d(np.arange(nq**3), chain)
    np.testing.assert_array_equal(g[others], others)  # lattice sites are a full spacing apart


def test_threshold_is_inclusive():
    nq, L, b = 4, 4.0, 0.25  # b^2 and the positions below are exact in FP32
    d = _place(nq, L, {5: (1.5, 0.5, 0.5), 9: (1.75, 0.5, 0.5)})
    assert fof.fof_groups(d, nq, L, b)[9] == 5
    d = _place(nq, L, {5: (1.5, 0.5, 0.5), 9: (1.75 + 2.0**-20, 0.5, 0.5)})
    assert fof.fof_groups(d, nq, L, b)[9] == 9


def test_lattice_translation_only_relabels():
    nq, L, b = 8, 8.0, 0.2
    d = _clumpy(7, nq, L)
    d = (np.round(d * 1024) / 1024).astype(np.float32)  # exact in FP32 after any integer shift
    g = fof.fof_groups(d, nq, L, b)
    t = (1, 2, 3)
    d4 = d.reshape(3, nq, nq, nq)
    ds = np.roll(d4, t, axis=(1, 2, 3)).reshape(3, -1)  # site q + t takes the displacement of q
    gs = fof.fof_groups(ds, nq, L, b)
    idx = np.arange(nq**3).reshape(nq, nq, nq)
    moved = np.roll(idx, t, axis=(0, 1, 2)).reshape(-1)  # new index -> old index
    # same partition: particles share a group before iff their images share one after
    np.testing.assert_array_equal(fof.canonical_labels(g[moved]), fof.canonical_labels(gs))


def test_groups_grow_with_the_linking_length():
    nq, L = 8, 8.0
    d = _clumpy(11, nq, L, spread=0.3)
    small, large = fof.fof_groups(d, nq, L, 0.15), fof.fof_groups(d, nq, L, 0.3)
    for r in np.unique(small):
        assert len(np.unique(large[small == r])) == 1
    assert len(np.unique(large)) < len(np.unique(small))


def test_labels_are_smallest_member_indices():
    nq, L = 8, 8.0
    g = fof.fof_groups(_clumpy(5, nq, L), nq, L, 0.2)
    assert np.all(g <= np.arange(nq**3))
    np.testing.assert_array_equal(g[g], g)


def _golden_masses():
    rows = {}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "paper_halo_masses.txt")
    for line in open(path):
        if line.strip() and not line.startswith("#"):
            f = line.split()
            rows[f[0]] = [float(x) for x in f[1:]]
    return rows


def test_particle_mass_and_warren_masses():
    g = _golden_masses()
    # Sec. 2.1: the MICE-GC particle mass; Sec. 2.5: the mass of the smallest kept halos
    om, L, n, value, tol = g["particle_mass"]
    mp = fof.particle_mass(om, L, int(n))
    assert mp == pytest.approx(value, rel=tol)
    om, L, n, members, value, tol = g["min_halo_log10_mass"]
    assert np.log10(fof.warren_mass(members, fof.particle_mass(om, L, int(n)))) == pytest.approx(value, abs=tol)
    # the correction removes one particle's worth at N = 1 and vanishes for large N
    assert fof.warren_mass(1, mp) == 0.0
    assert fof.warren_mass(1e8, mp) / (1e8 * mp) == pytest.approx(1.0, abs=2e-5)
    assert fof.warren_mass(1000, mp) < 1000 * mp


def test_catalog_and_mass_function():
    g = np.array([0, 0, 0, 3, 3, 5, 0, 3, 8, 8, 8, 8])
    roots, sizes = fof.halo_catalog(g, min_members=3)
    np.testing.assert_array_equal(roots, [0, 3, 8])
    np.testing.assert_array_equal(sizes, [4, 3, 4])
    # m_p = 1e10: N = 100 -> log10 M = 11.97 (below lo), 1000 -> 12.993, 10000 -> 13.998
    counts = fof.mass_function(np.array([100, 1000, 10000, 1000]), 1e10, 12.0, 1.0, 3)
    np.testing.assert_array_equal(counts, [2, 1, 0])


def test_brute_force_helper_sees_every_pair():
    # the brute force's own check: two particles exactly b apart across the boundary link
    nq, L, b = 4, 4.0, 0.25
    d = _place(nq, L, {0: (0.125, 0.5, 0.5), 1: (3.875, 0.5, 0.5)})
    g, _ = _brute_force(d, nq, L, b)
    assert g[1] == 0
    assert all(g[p] == p for p in range(2, nq**3))
    for p, q in itertools.combinations(range(2, 6), 2):
        assert g[p] != g[q]
