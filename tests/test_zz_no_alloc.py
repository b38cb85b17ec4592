"""cola_density_noalloc: the workspace-free density call, for callers that
cannot give the library scratch memory (their device memory is owned by their
own pool, or fully reserved by a running simulation).  Checked against the
ordinary workspace call on two calls in a row, through the C ABI; also the
largest accepted mesh, the rejected sizes, and the NaN output a non-finite
position gives, which must not leak into the next call."""
import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402
from synth import random_displacements  # noqa: E402


def _noalloc(cfg, d, out):
    fn = C.LIB.cola_density_noalloc
    fn.argtypes = [ctypes.POINTER(C.cola_config), ctypes.POINTER(C.cola_state), ctypes.c_void_p, ctypes.c_void_p]
    fn.restype = ctypes.c_int
    st = C.make_state(d)
    return fn(ctypes.byref(cfg), ctypes.byref(st), out.data_ptr(), torch.cuda.current_stream().cuda_stream)


def _check_twice(nq, ng, L, seed):
    cfg = C.make_config(nq, ng, L, 0.05)
    sim = C.Simulation(cfg)
    sim.init_tables()
    for call in range(2):
        d = torch.as_tensor(random_displacements(seed + 10 * call, nq, 0.7 * L / nq), device="cuda")
        sim.d.copy_(d)
        ref = sim.density()
        out = torch.full((ng, ng, ng), -7.0, dtype=torch.float32, device="cuda")
        assert _noalloc(cfg, sim.d, out) == 0
        torch.cuda.synchronize()
        # same kernels, same integer deposit: identical, well within the 3e-6 * m^3 density tolerance
        np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())
    return cfg, sim


def test_noalloc_density_matches_workspace_call_twice():
    for nq, ng, L, seed in ((32, 96, 128.0, 3), (16, 48, 64.0, 4)):
        _check_twice(nq, ng, L, seed)


def test_noalloc_density_at_the_largest_accepted_mesh():
    # ng = 128 fills the whole static array
    _check_twice(64, 128, 256.0, 5)


def test_noalloc_nonfinite_position_poisons_only_that_call():
    nq, ng, L = 16, 48, 64.0
    cfg = C.make_config(nq, ng, L, 0.05)
    sim = C.Simulation(cfg)
    sim.init_tables()
    d = torch.as_tensor(random_displacements(8, nq, 0.7 * L / nq), device="cuda")
    bad = d.clone()
    bad[1, 123] = float("nan")
    out = torch.zeros((ng, ng, ng), dtype=torch.float32, device="cuda")
    assert _noalloc(cfg, bad, out) == 0
    torch.cuda.synchronize()
    assert bool(torch.isnan(out).all())
    # the next clean call starts from cleared counts and a cleared flag
    sim.d.copy_(d)
    ref = sim.density()
    assert _noalloc(cfg, sim.d, out) == 0
    torch.cuda.synchronize()
    np.testing.assert_array_equal(out.cpu().numpy(), ref.cpu().numpy())


@pytest.mark.parametrize("nq,ng", [(64, 192), (26, 130), (48, 144), (8, 14)])
def test_noalloc_rejects_sizes(nq, ng):
    # beyond the static array (192, 144), or sizes cola_density rejects too (130 = 2 5 13, 14 = 2 7)
    cfg = C.make_config(nq, ng, 128.0, 0.05)
    d = torch.zeros((3, nq**3), dtype=torch.float32, device="cuda")
    out = torch.empty(1, dtype=torch.float32, device="cuda")
    assert _noalloc(cfg, d, out) == -3
