"""The largest run's 2304^3 mesh (768^3 particles, L = 1536 Mpc/h in the
benchmark).  Its 247 GB workspace leaves no room for a library-FFT reference,
so the force there is checked through properties that hold at any size."""
import pytest

torch = pytest.importorskip("torch")

from synth import random_displacements

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import dev  # noqa: E402


def test_2304_mesh_force_is_momentum_conserving_and_translation_covariant():
    # the largest run's mesh (247 GB of workspace leaves no room for the library
    # reference): 256^3 particles, 9 cells per spacing
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
