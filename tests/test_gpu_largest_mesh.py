"""The largest run's 2304^3 mesh (768^3 particles, L = 1536 Mpc/h in the
benchmark).  Its workspace leaves no room for a library-FFT reference; the
force there is checked element by element against the FP64 oracle on inputs
whose exact force it can compute on a reduced periodic cell (a lattice
displaced along one axis), and through properties that hold at any size."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import pm
from synth import random_displacements

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev  # noqa: E402


def test_2304_mesh_force_of_a_displaced_lattice_vs_oracle_every_particle():
    # 256^3 particles on the 2304^3 mesh (9 cells per spacing), L = 1536 Mpc/h:
    # the lattice displaced along x, then y, then z, by a seeded amount that
    # depends only on the lattice index along that axis; every particle's force
    # against the oracle's exact value (lattice_wave_force), rel-L2 <= 1e-5
    nq, ng, box, a = 256, 2304, 1536.0, 0.5
    green = 1.5 * 0.25 / a
    s = C.Simulation(C.make_config(nq, ng, box, 0.05))
    s.init_tables()
    lat = np.arange(nq)
    try:
        for axis in range(3):
            dline = (np.random.default_rng(40 + axis).standard_normal(nq) * 0.6 * box / nq).astype(np.float32)
            d = torch.zeros((3, nq, nq, nq), dtype=torch.float32, device="cuda")
            shape = [1, 1, 1]
            shape[axis] = nq
            d[axis] = dev(dline).view(shape)
            s.d.copy_(d.reshape(3, -1))
            f = s.force(a).cpu().numpy().astype(np.float64)
            assert s.status() == 0
            ref = pm.lattice_wave_force(dline.astype(np.float64), nq, ng, box, green, axis)
            rel = np.linalg.norm(f - ref) / np.linalg.norm(ref)
            assert rel <= 1e-5, (axis, rel)
            del ref, f
    finally:
        del s
        torch.cuda.empty_cache()


def test_2304_mesh_force_is_momentum_conserving_and_translation_covariant():
    # random displacements: 256^3 particles, 9 cells per spacing
    nq, ng, box, a = 256, 2304, 2304.0, 0.5
    s = C.Simulation(C.make_config(nq, ng, box, 0.05))
    s.init_tables()
    s.d.copy_(dev(random_displacements(9, nq, 0.7 * box / nq)))
    f = s.force(a).clone()
    assert s.status() == 0
    assert f.double().sum(dim=1).abs().max().item() < 1e-6 * f.double().abs().sum(dim=1).max().item()
    d = s.d.view(3, nq, nq, nq)
    s.d.copy_(torch.roll(d, shifts=1, dims=2).reshape(3, -1))
    f2 = s.force(a)
    f_ref = torch.roll(f.view(3, nq, nq, nq), shifts=1, dims=2).reshape(3, -1)
    rel = (torch.linalg.norm(f2 - f_ref) / torch.linalg.norm(f_ref)).item()
    del s
    torch.cuda.empty_cache()
    assert rel < 1e-5
