"""Philox-4x32-10 counter-based RNG and the Gaussian white noise of the initial
conditions.

Test infrastructure only (see ``oracle/__init__``).

The paper only says the initial conditions are random Gaussian fields drawn with
a fixed seed shared by all runs (Sec. 2.2, Sec. 2.3).  Reading adopted so that
CPU and GPU draw the same noise without sharing code: each side implements
Philox-4x32 with 10 rounds from its published definition (Salmon, Moraes, Dror
& Shaw 2011, "Parallel random numbers: as easy as 1, 2, 3", SC'11):

  round:  (hi0, lo0) = mulhilo(0xD2511F53, c0); (hi1, lo1) = mulhilo(0xCD9E8D57, c2)
          c = (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0)
  key schedule between rounds: k0 += 0x9E3779B9, k1 += 0xBB67AE85.

Noise of Lagrangian cell n (C order, z fastest) uses key = (seed & 0xffffffff,
seed >> 32) and counter = (n & 0xffffffff, n >> 32, 0, 0).  The four output
words give two 53-bit uniforms on (0, 1]:
  u = ((w_a >> 5) * 2^26 + (w_b >> 6) + 1) * 2^-53,  u1 from (w0, w1), u2 from (w2, w3)
and one normal deviate by the Box-Muller cosine branch
  g = sqrt(-2 ln u1) cos(2 pi u2).

Pin: the published Philox-4x32-10 known-answer vectors
(tests/golden/philox4x32_10_kat.txt) and the first two moments of the normal.
"""
from __future__ import annotations

import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = np.uint64(0x9E3779B9)
W1 = np.uint64(0xBB67AE85)
MASK32 = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: (4, n) uint32-valued, key: (2, n) or (2,) uint32-valued.
    Returns the (4, n) uint32 output block."""
    c = [np.asarray(x, dtype=np.uint64) & MASK32 for x in ctr]
    k0 = np.asarray(key[0], dtype=np.uint64) & MASK32
    k1 = np.asarray(key[1], dtype=np.uint64) & MASK32
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK32
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK32
        c = [hi1 ^ c[1] ^ k0, lo1, hi0 ^ c[3] ^ k1, lo0]
    return np.stack([x.astype(np.uint32) for x in c])


def uniform53(w_a, w_b):
    """Two 32-bit words -> a 53-bit uniform on (0, 1]."""
    a = np.asarray(w_a, dtype=np.uint64) >> np.uint64(5)
    b = np.asarray(w_b, dtype=np.uint64) >> np.uint64(6)
    m = a * np.uint64(1 << 26) + b + np.uint64(1)
    return m.astype(np.float64) * 2.0**-53


def white_noise(seed: int, n_cells: int, first: int = 0) -> np.ndarray:
    """Unit-variance Gaussian deviates for cells first .. first+n_cells-1."""
    idx = np.arange(first, first + n_cells, dtype=np.uint64)
    ctr = [idx & MASK32, idx >> np.uint64(32), np.zeros_like(idx), np.zeros_like(idx)]
    key = (np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    w = philox4x32_10(ctr, key)
    u1 = uniform53(w[0], w[1])
    u2 = uniform53(w[2], w[3])
    return np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)


def white_noise_grid(seed: int, nq: int) -> np.ndarray:
    """The (nq, nq, nq) white-noise field on the Lagrangian grid (C order)."""
    return white_noise(seed, nq**3).reshape(nq, nq, nq)
