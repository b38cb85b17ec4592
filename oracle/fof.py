"""Friends-of-friends halo finder and halo mass function (Sec. 2.1: FoF of
Davis et al. 1985, linking length b = 0.2; Sec. 2.5: halos of more than
100 particles, i.e. at least 101, masses with the Warren et al. 2006 correction
M = m_p N (1 - N^-0.6)).

Test infrastructure only (see ``oracle/__init__``).

Readings:
* The linking length is b times the mean inter-particle spacing L / nq (b = 0.2
  in the paper).  Positions are taken in units of that spacing,
  s = q + d nq / L for lattice site q and displacement d, periodic in [0, nq).
* Two particles are friends when their minimum-image separation is at most b
  (<=); the groups are the connected components of the friendship graph.
* That decision fixes an integer result (the partition), so it is taken in
  FP32 with the formula the CUDA path uses, each operation rounded once:
    u = float32(q) + float32(d) * float32(nq / L), wrapped into [0, nq) by
        u - nq floor(u / nq), then u < 0 -> u + nq, then u >= nq -> u - nq
        (the last two undo the division's rounding; in this order the result
        always lies in [0, nq));
    delta = u_p - u_q, brought to the minimum image by one +-nq when
        |delta| > nq / 2;
    r2 = (dx dx + dy dy) + dz dz;  friends iff r2 <= float32(b * b).
  Everything else (the components, the masses, the histogram) is exact or FP64.
* A group is labelled by the smallest particle index in it.
* Particle mass m_p = rho_c Omega_m (L / nq)^3 in Msun/h (L in Mpc/h), with
  rho_c = 3 H0^2 / (8 pi G) = 2.77536627e11 h^2 Msun Mpc^-3.
* Mass function: halo counts in bins of log10(M / (Msun/h)); bin
  i = floor((log10 M - lo) / dlog), kept when 0 <= i < nbins (FP64).

Pins (tests/test_oracle_fof.py): an O(N^2) brute force with a plain
union-find; chains across the periodic boundary just inside and just outside
the linking length; the exact threshold; relabelling under a lattice
translation; monotonicity in b; the Warren mass closed form and the MICE-GC
particle mass the paper prints (2.93e10 Msun/h).
"""
from __future__ import annotations

import numpy as np
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components
from scipy.spatial import cKDTree

RHO_CRIT = 2.77536627e11  # h^2 Msun / Mpc^3


def lattice_sites(nq: int) -> np.ndarray:
    """(3, nq^3) int64 lattice indices (i, j, k) of particle p = (i nq + j) nq + k."""
    p = np.arange(nq**3, dtype=np.int64)
    return np.stack([p // (nq * nq), (p // nq) % nq, p % nq])


def wrapped_positions(d, nq: int, L: float) -> np.ndarray:
    """FP32 positions in units of the mean spacing, wrapped into [0, nq)."""
    d = np.asarray(d, dtype=np.float32).reshape(3, -1)
    inv = np.float32(nq / L)
    nqf = np.float32(nq)
    u = lattice_sites(nq).astype(np.float32) + d * inv
    u = u - nqf * np.floor(u / nqf)
    u = np.where(u < np.float32(0), u + nqf, u)
    u = np.where(u >= nqf, u - nqf, u)
    return u.astype(np.float32)


def separation2(up: np.ndarray, uq: np.ndarray, nq: int) -> np.ndarray:
    """FP32 squared minimum-image separation of positions up, uq (3, ...)."""
    nqf = np.float32(nq)
    half = np.float32(nq / 2)
    dl = (up - uq).astype(np.float32)
    dl = np.where(dl > half, dl - nqf, dl)
    dl = np.where(dl < -half, dl + nqf, dl)
    dl = dl.astype(np.float32)
    return ((dl[0] * dl[0] + dl[1] * dl[1]) + dl[2] * dl[2]).astype(np.float32)


def linked(up, uq, nq: int, b: float):
    return separation2(up, uq, nq) <= np.float32(b * b)


def canonical_labels(comp: np.ndarray) -> np.ndarray:
    """Relabel a component numbering by the smallest member index."""
    n = comp.size
    first = np.full(comp.max() + 1, n, dtype=np.int64)
    np.minimum.at(first, comp, np.arange(n, dtype=np.int64))
    return first[comp]


def fof_groups(d, nq: int, L: float, b: float = 0.2) -> np.ndarray:
    """Group label (smallest member index) of every particle.

    Candidate pairs come from a periodic k-d tree query with a radius a little
    above b (a superset); the FP32 rule above decides which of them are friends,
    and the connected components of the resulting graph are the groups."""
    u = wrapped_positions(d, nq, L)
    n = u.shape[1]
    pts = np.ascontiguousarray(u.T.astype(np.float64))
    pairs = cKDTree(pts, boxsize=float(nq)).query_pairs(b + 1e-3, output_type="ndarray")
    if pairs.size:
        keep = linked(u[:, pairs[:, 0]], u[:, pairs[:, 1]], nq, b)
        pairs = pairs[keep]
    g = coo_matrix((np.ones(len(pairs), dtype=np.int8), (pairs[:, 0], pairs[:, 1])), shape=(n, n))
    _, comp = connected_components(g, directed=False)
    return canonical_labels(comp)


def particle_mass(omega_m: float, L: float, nq: int) -> float:
    """m_p in Msun/h for a box of side L Mpc/h holding nq^3 particles."""
    return RHO_CRIT * omega_m * (L / nq) ** 3


def warren_mass(n, m_p: float):
    """M = m_p N (1 - N^-0.6) (Warren et al. 2006)."""
    n = np.asarray(n, dtype=np.float64)
    return m_p * n * (1.0 - n ** -0.6)


def halo_catalog(group: np.ndarray, min_members: int = 101):
    """(root, size) of every group with at least min_members particles, by root."""
    roots, sizes = np.unique(group, return_counts=True)
    keep = sizes >= min_members
    return roots[keep].astype(np.int64), sizes[keep].astype(np.int64)


def mass_function(sizes, m_p: float, lo: float, dlog: float, nbins: int) -> np.ndarray:
    """Halo counts per bin of log10 M (Warren masses)."""
    lm = np.log10(warren_mass(sizes, m_p))
    i = np.floor((lm - lo) / dlog).astype(np.int64)
    i = i[(i >= 0) & (i < nbins)]
    return np.bincount(i, minlength=nbins).astype(np.int64)
