"""Seeded synthetic inputs (NumPy Generator draws), returned as float32 arrays in
the library's layout: particle fields are SoA (3, nq^3) in Lagrangian C order."""
from __future__ import annotations

import numpy as np

__all__ = ["random_displacements", "random_state", "plane_wave_psi1", "crossed_waves_delta",
           "random_mesh", "single_mode_delta", "clumpy_displacements"]


def random_displacements(seed: int, nq: int, rms: float) -> np.ndarray:
    """Gaussian displacements of the given rms (Mpc/h) per component."""
    rng = np.random.default_rng(seed)
    return (rng.standard_normal((3, nq**3)) * rms).astype(np.float32)


def random_state(seed: int, nq: int, rms_d: float, rms_v: float, rms_psi: float):
    """A state dict (d, v, psi1, psi2) of independent Gaussian fields."""
    rng = np.random.default_rng(seed)
    f = lambda s: (rng.standard_normal((3, nq**3)) * s).astype(np.float32)
    return {"d": f(rms_d), "v": f(rms_v), "psi1": f(rms_psi), "psi2": f(0.1 * rms_psi)}


def plane_wave_psi1(nq: int, L: float, amp: float, mode: int = 1) -> np.ndarray:
    """Zel'dovich displacement of delta = amp cos(k q_x), k = 2 pi mode / L:
    Psi1_x = -(amp/k) sin(k q_x), other components zero (3, nq^3)."""
    k = 2.0 * np.pi * mode / L
    i = np.arange(nq)
    qx = np.broadcast_to((i * (L / nq))[:, None, None], (nq, nq, nq)).reshape(-1)
    out = np.zeros((3, nq**3))
    out[0] = -(amp / k) * np.sin(k * qx)
    return out


def crossed_waves_delta(n: int, L: float, A: float, B: float, mode: int = 1) -> np.ndarray:
    """delta(q) = A cos(k x) + B cos(k y) on an n^3 grid, k = 2 pi mode / L."""
    k = 2.0 * np.pi * mode / L
    x = np.arange(n) * (L / n)
    return (A * np.cos(k * x)[:, None, None] + B * np.cos(k * x)[None, :, None]
            + 0.0 * x[None, None, :])


def single_mode_delta(n: int, L: float, eps: float, nvec) -> np.ndarray:
    """delta = eps cos(k . x) on the mesh nodes, k = 2 pi nvec / L."""
    x = np.arange(n) * (L / n)
    kx, ky, kz = (2.0 * np.pi * np.asarray(nvec) / L)
    return eps * np.cos(kx * x[:, None, None] + ky * x[None, :, None] + kz * x[None, None, :])


def random_mesh(seed: int, shape, scale: float = 1.0) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return (rng.standard_normal(shape) * scale).astype(np.float32)


def clumpy_displacements(seed: int, nq: int, L: float, nclump: int, spread: float, frac: float = 0.7) -> np.ndarray:
    """Displacements (3, nq^3) that move a fraction `frac` of the particles into
    nclump Gaussian clumps of rms `spread` (in mean spacings) around uniform
    random centres; the rest stay within 0.05 spacings of their lattice sites."""
    rng = np.random.default_rng(seed)
    p = np.arange(nq**3, dtype=np.int64)
    q = np.stack([p // (nq * nq), (p // nq) % nq, p % nq]).astype(np.float64)
    centres = rng.uniform(0, nq, (nclump, 3))
    target = q + rng.normal(0.0, 0.05, q.shape)
    moved = rng.uniform(size=nq**3) < frac
    which = rng.integers(0, nclump, moved.sum())
    target[:, moved] = centres[which].T + rng.normal(0.0, spread, (3, moved.sum()))
    return ((target - q) * (L / nq)).astype(np.float32)
