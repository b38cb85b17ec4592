"""Particle-mesh force: CIC deposit, Poisson solve with the k-space Green's
function and ik gradient, CIC gather (Sec. 2.2: PM with a mesh PM_grid times
finer than the particle grid, one forward and three inverse FFTs per step).

Test infrastructure only (see ``oracle/__init__``).

Readings (the paper prints none of these formulas):

* Particle p with Lagrangian index (i, j, k) and displacement d sits at mesh
  coordinate u = (i, j, k) * ng/nq + 1/2 + d * ng / L, periodic: the
  Lagrangian lattice is translated by half a mesh cell so that unperturbed
  particles sit at cell midpoints.  (A global translation changes nothing
  physical in a periodic box; on the nodes themselves the CIC weight has a
  kink and a slightly displaced lattice responds with |d| instead of d.)
* CIC: weight (1 - |s|) for |s| < 1 per axis to the two nearest nodes,
  node c at position c * L/ng.  Every particle has unit mass, so the mean
  count per cell is (nq/ng)^3 and delta = rho * (ng/nq)^3 - 1.
* Poisson: lap Phi = 3/2 Om/a delta (units H0 = 1, x in Mpc/h), solved with
  the continuous -1/k^2 kernel: Phi_k = -green delta_k / k^2, green = 3/2 Om/a,
  Phi_0 = 0.
* Force F = -grad Phi: F_j,k = -i k_j Phi_k, with k_j := 0 on the Nyquist
  plane of axis j (keeps F real).  No CIC deconvolution, no smoothing.
* Gather with the same CIC kernel as the deposit (momentum conserving).

Pins (tests/test_oracle_pm.py): sum of the CIC mesh = particle count; a
particle on a node fills one cell; the net force on all particles vanishes;
a prescribed single Fourier mode gives the closed-form force; a single
particle's force matches the periodic point-mass (Ewald) force beyond a few
cells; direct DFT vs numpy FFT; lattice_wave_force equals pm_force on whole
meshes with m = 1 .. 4 cells per spacing along each axis.
"""
from __future__ import annotations

import numpy as np

from .lpt import _irfftn, _rfftn, kgrid


def lagrangian_index(nq: int):
    """(3, nq^3) integer Lagrangian coordinates in particle (C) order."""
    i = np.arange(nq)
    g = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([x.reshape(-1) for x in g])


def mesh_coords(d: np.ndarray, nq: int, ng: int, L: float) -> np.ndarray:
    """Mesh coordinates u (3, Np) in [0, ng) of displaced particles."""
    u = lagrangian_index(nq) * (ng / nq) + 0.5 + np.asarray(d, dtype=np.float64) * (ng / L)
    return np.mod(u, ng)


def cic_weights(u: np.ndarray, ng: int):
    """Yields (flat cell index, weight) for the 8 CIC corners of each particle."""
    c0 = np.floor(u).astype(np.int64)
    f = u - c0
    for dx in (0, 1):
        wx = f[0] if dx else 1.0 - f[0]
        ix = (c0[0] + dx) % ng
        for dy in (0, 1):
            wy = f[1] if dy else 1.0 - f[1]
            iy = (c0[1] + dy) % ng
            for dz in (0, 1):
                wz = f[2] if dz else 1.0 - f[2]
                iz = (c0[2] + dz) % ng
                yield (ix * ng + iy) * ng + iz, wx * wy * wz


def cic_deposit(u: np.ndarray, ng: int, weights=None) -> np.ndarray:
    """Mass on the ng^3 mesh (each particle mass 1 unless weights given)."""
    rho = np.zeros(ng**3)
    mass = 1.0 if weights is None else np.asarray(weights, dtype=np.float64)
    for idx, w in cic_weights(u, ng):
        rho += np.bincount(idx, weights=w * mass, minlength=ng**3)
    return rho.reshape(ng, ng, ng)


def cic_gather(mesh: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Interpolate a (ng, ng, ng) field to the particles."""
    ng = mesh.shape[0]
    flat = mesh.reshape(-1)
    out = np.zeros(u.shape[1])
    for idx, w in cic_weights(u, ng):
        out += w * flat[idx]
    return out


def density_contrast(d, nq: int, ng: int, L: float) -> np.ndarray:
    """delta = rho (ng/nq)^3 - 1 on the ng^3 mesh."""
    u = mesh_coords(d, nq, ng, L)
    return cic_deposit(u, ng) * (ng / nq) ** 3 - 1.0


def radial_filter(kmag: np.ndarray, T: np.ndarray, kmax: float) -> np.ndarray:
    """Piecewise-linear transfer function on nodes b * kmax / (len(T) - 1)
    (the learned coarse-mesh filter; not in the paper)."""
    nb = len(T)
    u = kmag / (kmax / (nb - 1))
    b = np.minimum(np.floor(u).astype(np.int64), nb - 2)
    f = np.minimum(u - b, 1.0)
    return (1.0 - f) * T[b] + f * T[b + 1]


def force_mesh_from_delta(delta: np.ndarray, L: float, green: float, filt=None) -> np.ndarray:
    """(3, ng, ng, ng) force field F = -grad Phi, lap Phi = green * delta; with
    filt = T (node values) the potential is multiplied by the radial filter,
    nodes spaced sqrt(3) pi ng / L / (len(T) - 1)."""
    ng = delta.shape[0]
    kx, ky, kz, nx, ny, nz = kgrid(ng, L)
    k2 = kx**2 + ky**2 + kz**2
    k2[0, 0, 0] = 1.0
    dk = _rfftn(delta)
    phik = -green * dk / k2
    if filt is not None:
        phik = phik * radial_filter(np.sqrt(k2), np.asarray(filt, dtype=np.float64), np.sqrt(3.0) * np.pi * ng / L)
    phik[0, 0, 0] = 0.0
    out = []
    for kj, nyq in ((kx, nx), (ky, ny), (kz, nz)):
        kd = np.where(nyq, 0.0, kj)
        out.append(_irfftn(-1j * kd * phik, delta.shape))
    return np.stack(out)


def pm_force(d, nq: int, ng: int, L: float, green: float):
    """Force on every particle (3, Np): deposit, Poisson + gradient, gather."""
    u = mesh_coords(d, nq, ng, L)
    delta = cic_deposit(u, ng) * (ng / nq) ** 3 - 1.0
    fm = force_mesh_from_delta(delta, L, green)
    return np.stack([cic_gather(fm[j], u) for j in range(3)])


def lattice_wave_force(dline, nq: int, ng: int, L: float, green: float, axis: int = 0) -> np.ndarray:
    """The force (3, Np) that pm_force gives for the Lagrangian lattice displaced
    along one axis only, by an amount that depends only on the lattice index
    along that axis: d_axis(p) = dline[i_axis(p)], the other components zero.

    Same readings as pm_force, computed exactly on a smaller periodic cell: with
    m = ng / nq an integer, the lattice repeats every m cells across the axis,
    so the density, the potential and the force repeat too, and only the modes
    whose transverse indices are multiples of nq are present.  Those are the
    modes of an ng x m x m mesh whose cells keep the size L / ng (transverse
    wavenumbers 2 pi n / (m L / ng)); a transverse index n = +-m/2 there is the
    full mesh's Nyquist plane.  Every particle of one line sits at the same
    place in that cell (transverse mesh coordinate 1/2), so one line of nq
    particles gives everyone's force."""
    if ng % nq:
        raise ValueError("needs ng a multiple of nq")
    m = ng // nq
    dline = np.asarray(dline, dtype=np.float64)
    u = np.mod(np.arange(nq) * m + 0.5 + dline * (ng / L), ng)
    shape = (ng, m, m)
    c0 = np.floor(u).astype(np.int64)
    f = u - c0
    rho = np.zeros(shape)
    for dx in (0, 1):
        wx = f if dx else 1.0 - f
        ix = (c0 + dx) % ng
        for iy in (0, 1 % m):
            for iz in (0, 1 % m):
                np.add.at(rho, (ix, iy, iz), 0.25 * wx)
    delta = rho * (ng / nq) ** 3 - 1.0
    dk = np.fft.rfftn(delta)
    nx = np.fft.fftfreq(ng, d=1.0 / ng)[:, None, None]
    nt = np.fft.fftfreq(m, d=1.0 / m)[None, :, None]
    nh = np.arange(m // 2 + 1, dtype=np.float64)[None, None, :]
    cell = L / ng
    kx = 2.0 * np.pi * nx / L
    ky = 2.0 * np.pi * nt / (m * cell)
    kz = 2.0 * np.pi * nh / (m * cell)
    k2 = kx**2 + ky**2 + kz**2
    k2[0, 0, 0] = 1.0
    phik = -green * dk / k2
    phik[0, 0, 0] = 0.0
    even = m % 2 == 0
    kdx = np.where(np.abs(nx) == ng // 2, 0.0, kx)
    kdy = np.where(even & (np.abs(nt) == m // 2), 0.0, ky)
    kdz = np.where(even & (nh == m // 2), 0.0, kz)
    line = np.zeros((3, nq))
    for j, kd in enumerate((kdx, kdy, kdz)):
        fm = np.fft.irfftn(-1j * kd * phik, s=shape, axes=(0, 1, 2))
        # gather: weights 1/2 to transverse cells 0 and 1 on both transverse axes
        for dx in (0, 1):
            wx = f if dx else 1.0 - f
            ix = (c0 + dx) % ng
            for iy in (0, 1 % m):
                for iz in (0, 1 % m):
                    line[j] += 0.25 * wx * fm[ix, iy, iz]
    # the axis-0 cell's components (along, across, across) -> the lattice's axes
    comp = [1, 2]
    comp.insert(axis, 0)
    idx = np.arange(nq)
    lat = np.meshgrid(idx, idx, idx, indexing="ij")[axis].reshape(-1)
    return np.stack([line[comp[c]][lat] for c in range(3)])
