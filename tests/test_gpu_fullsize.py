"""Checks at the benchmarked size (512^3 particles, 1536^3 mesh, L = 1536
Mpc/h, the launch configuration bench.py times): sampled outputs against the
oracle where it can compute them, and properties that hold at any size."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import cosmology as cm
from oracle import lpt

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import host  # noqa: E402

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
