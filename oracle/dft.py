"""Direct O(N^2) discrete Fourier transforms, used only to pin numpy's FFT
(which the oracle uses as a library step) on tiny and mixed-radix shapes.

Test infrastructure only (see ``oracle/__init__``).

X[k] = sum_n x[n] exp(-2 pi i k n / N) along each axis in turn, with the
angle reduced modulo N in integers before the cosine/sine so the FP64
result is accurate to a few ulp.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(n: int, sign: int = -1) -> np.ndarray:
    k = np.arange(n)
    kn = np.outer(k, k) % n
    ang = 2.0 * np.pi * kn / n
    return np.cos(ang) + sign * 1j * np.sin(ang)


def dftn(x: np.ndarray, sign: int = -1) -> np.ndarray:
    """Full complex DFT over every axis."""
    out = np.asarray(x, dtype=np.complex128)
    for ax in range(out.ndim):
        m = dft_matrix(out.shape[ax], sign)
        out = np.moveaxis(np.tensordot(m, np.moveaxis(out, ax, 0), axes=(1, 0)), 0, ax)
    return out


def rdftn(x: np.ndarray) -> np.ndarray:
    """Half spectrum (last axis 0..N/2) of the forward DFT of a real array."""
    full = dftn(x, -1)
    return full[..., : x.shape[-1] // 2 + 1]
