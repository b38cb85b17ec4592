"""Checks at the benchmarked size (512^3 particles, 1536^3 mesh, L = 1536
Mpc/h, the launch configuration bench.py times) and at 256^3 / 768^3: sampled
outputs against the oracle where it can compute them, properties that hold at
any size, and the whole force against the same PM force written with torch's
library FFT (a cross-check independent of this package's kernels)."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cosmology as cm
from oracle import lpt
from synth import random_displacements

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev, host  # noqa: E402

NQ, NG, L = 512, 1536, 1536.0
COSMO = cm.Cosmology()


@pytest.fixture(scope="module")
def sim():
    s = C.Simulation(C.make_config(NQ, NG, L, 0.05))
    s.ic(seed=1)
    yield s
    del s
    torch.cuda.empty_cache()


def test_fullsize_2lpt_fields_on_sampled_particles(sim):
    # full FP64 oracle field (threaded pocketfft), compared on 20000 particles
    lpt.FFT_WORKERS = max(1, os.cpu_count() or 1)
    try:
        g = cm.Growth(COSMO)
        D1, _, D2, _ = g(np.array([0.05]))
        ref = lpt.initial_conditions(1, NQ, L, cm.LinearPower(COSMO), D1[0], D2[0])
    finally:
        lpt.FFT_WORKERS = 1
    idx = np.random.default_rng(0).choice(NQ**3, 20000, replace=False)
    it = torch.as_tensor(idx, device="cuda")
    for key in ("psi1", "psi2", "d"):
        got = host(getattr(sim, key)[:, it])
        want = ref[key][:, idx]
        err = np.linalg.norm(got - want) / np.linalg.norm(want)
        assert err < 1e-5, (key, err)


def test_fullsize_force_conserves_momentum_and_is_translation_covariant(sim):
    a = 0.3
    f = sim.force(a).clone()
    assert sim.status() == 0
    net = f.double().sum(dim=1).abs().max().item()
    assert net < 1e-6 * f.double().abs().sum(dim=1).max().item()
    # shift the whole particle lattice by one spacing along x: the density moves
    # by NG/NQ = 3 mesh cells and every particle feels its neighbour's old force
    d = sim.d.view(3, NQ, NQ, NQ)
    saved = sim.d.clone()
    sim.d.copy_(torch.roll(d, shifts=1, dims=1).reshape(3, -1))
    f2 = sim.force(a)
    f_ref = torch.roll(f.view(3, NQ, NQ, NQ), shifts=1, dims=1).reshape(3, -1)
    rel = (torch.linalg.norm(f2 - f_ref) / torch.linalg.norm(f_ref)).item()
    sim.d.copy_(saved)
    assert rel < 1e-5


def test_fullsize_unperturbed_lattice_feels_no_force():
    s = C.Simulation(C.make_config(NQ, NG, L, 0.05))
    s.init_tables()
    f = s.force(0.5)
    assert f.abs().max().item() < 1e-4  # the CIC lattice is exactly uniform: FFT round-off only
    del s
    torch.cuda.empty_cache()


def torch_pm_force(d, nq, ng, L, green, chunk=1 << 23):
    """The PM force of the oracle (CIC deposit, continuous Green's function,
    spectral gradient with k_j = 0 on axis j's Nyquist plane, CIC gather),
    written with torch tensor ops and torch.fft: FP64 particle coordinates,
    FP32 meshes.  Test-only cross-check at sizes the FP64 oracle cannot hold."""
    dv = d.device
    npart = nq**3

    def corners(p0, p1):
        p = torch.arange(p0, p1, device=dv, dtype=torch.int64)
        q = torch.stack([p // (nq * nq), (p // nq) % nq, p % nq]).double()
        u = torch.remainder(q * (ng / nq) + 0.5 + d[:, p0:p1].double() * (ng / L), ng)
        c0 = torch.floor(u)
        f = u - c0
        c0 = c0.long()
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    w = (f[0] if dx else 1 - f[0]) * (f[1] if dy else 1 - f[1]) * (f[2] if dz else 1 - f[2])
                    idx = (((c0[0] + dx) % ng) * ng + (c0[1] + dy) % ng) * ng + (c0[2] + dz) % ng
                    yield idx, w

    rho = torch.zeros(ng**3, dtype=torch.float32, device=dv)
    for p0 in range(0, npart, chunk):
        for idx, w in corners(p0, min(npart, p0 + chunk)):
            rho.index_add_(0, idx, w.float())
    delta = rho.view(ng, ng, ng)
    delta.mul_((ng / nq) ** 3).sub_(1.0)
    dk = torch.fft.rfftn(delta)
    del rho, delta
    kf = 2 * np.pi / L
    n_full = torch.fft.fftfreq(ng, 1.0 / ng, device=dv)
    n_half = torch.fft.rfftfreq(ng, 1.0 / ng, device=dv)
    kx = (kf * n_full).float().view(-1, 1, 1)
    ky = (kf * n_full).float().view(1, -1, 1)
    kz = (kf * n_half).float().view(1, 1, -1)
    k2 = kx * kx + ky * ky + kz * kz
    k2[0, 0, 0] = 1.0
    phik = dk.mul_(-green).div_(k2)
    del k2
    phik[0, 0, 0] = 0.0
    out = torch.zeros((3, npart), dtype=torch.float64, device=dv)
    for j, kj in enumerate((kx, ky, kz)):
        kd = kj.clone()
        kd.view(-1)[ng // 2] = 0.0  # Nyquist plane of axis j
        fj = torch.fft.irfftn(phik * (-1j * kd), s=(ng, ng, ng)).reshape(-1)
        for p0 in range(0, npart, chunk):
            acc = torch.zeros(min(npart, p0 + chunk) - p0, dtype=torch.float64, device=dv)
            for idx, w in corners(p0, min(npart, p0 + chunk)):
                acc += w * fj[idx].double()
            out[j, p0:p0 + acc.numel()] = acc
        del fj
    return out


# (nq, ng, L, column widths of the strided and fused passes; 0 = built-in)
@pytest.mark.parametrize("nq,ng,L,widths", [(256, 768, 768.0, (0,)), (384, 1152, 1152.0, (0,)),
                                            (NQ, NG, L, (0, 4))])
def test_force_matches_library_fft_reference(nq, ng, L, widths):
    a = 0.5
    d = dev(random_displacements(5, nq, 0.7 * L / nq))
    s = C.Simulation(C.make_config(nq, ng, L, 0.05))
    s.init_tables()
    s.d.copy_(d)
    got = []
    try:
        for B in widths:
            C.cola_fft_set_tile(ng, B)
            got.append(s.force(a).double().cpu())
            assert s.status() == 0
    finally:
        C.cola_fft_set_tile(ng, 0)
    del s
    torch.cuda.empty_cache()
    ref = torch_pm_force(d, nq, ng, L, 1.5 * COSMO.omega_m / a).cpu()
    for B, g in zip(widths, got):
        rel = (torch.linalg.norm(g - ref) / torch.linalg.norm(ref)).item()
        assert rel < 1e-5, (B, rel)

