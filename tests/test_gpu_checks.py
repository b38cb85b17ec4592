"""The bounds-checked build of the library (COLA_CHECKS defined).

It stands in for a memory checker, which cannot run here: every data-dependent
index of the PM step (bin key, sorted position, the z cell of a CIC record) is
checked on the device before the access it guards, and a failed check skips the
access and latches COLA_EBOUNDS.  A child process loads that build and runs the
tiny and odd-shape cases (2LPT set-up, PM force, two COLA nodes, density) on
both PM paths:
the results must be bit-identical to the normal build's and the status word
clear.  The probe hook shows the latch itself: an index that fails its check
leaves COLA_EBOUNDS in the status word, with the write skipped.
"""
import hashlib
import importlib.util
import os
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TESTS = os.path.join(ROOT, "tests")

# (nq, ng, L): tiny, odd radices (3, 5), ng = nq, a mesh of 1.5 nq, the
# largest runtime-path shape of the parity suite, and a 768^3 mesh (the
# warp-row fused passes)
CASES = [(16, 48, 64.0), (10, 30, 40.0), (12, 18, 48.0), (6, 18, 30.0), (8, 12, 40.0), (16, 16, 64.0),
         (64, 192, 192.0), (128, 768, 768.0)]


PATHS = (1, 2)  # fused passes, separate kernels (cola_pm_set_path)


def outputs(nq, ng, L, path):
    """2LPT set-up, PM force, two COLA nodes and the density with the library
    this process loaded, on one PM path, and the status word after them."""
    assert C.LIB.cola_pm_set_path(path) == 0
    try:
        sim = C.Simulation(C.make_config(nq, ng, L, 0.05, 1.0, 40))
        sim.ic(seed=9)
        out = {"force": digest(sim.force(0.05))}
        sim.step(0)
        sim.step(1)
        out.update(d=digest(sim.d), v=digest(sim.v), density=digest(sim.density()), status=np.array([sim.status()]))
    finally:
        C.LIB.cola_pm_set_path(0)
    return out


def digest(t):
    """SHA-256 of a tensor's bytes: equal digests mean bit-identical arrays."""
    return np.frombuffer(hashlib.sha256(t.contiguous().cpu().numpy().tobytes()).digest(), dtype=np.uint8)


def probe():
    """(launch rc, status after it) of the probe hook, for indexes inside and
    outside the checked bound n, on the workspace of a small initialised
    simulation (cola_init clears its status word)."""
    sim = C.Simulation(C.make_config(8, 16, 32.0, 0.05, 1.0, 4))
    sim.init_tables()
    ws = sim.ws
    s = torch.cuda.current_stream().cuda_stream
    res = []
    for index, n in ((3, 8), (8, 8), (63, 64), (40, 7)):
        rc = C.LIB.cola_checks_probe(index, n, ws.data_ptr(), ws.numel(), s)
        res.append((rc, C.LIB.cola_status(ws.data_ptr(), ws.numel(), s)))
    return res


def child(path):
    assert C.LIB.cola_checks_enabled() == 1, "the child must load the checked build"
    out = {f"{nq}_{ng}_{p}_{k}": v for nq, ng, L in CASES for p in PATHS for k, v in outputs(nq, ng, L, p).items()}
    out["probe"] = np.array(probe())
    np.savez(path, **out)


@pytest.fixture(scope="module")
def checked(tmp_path_factory):
    spec = importlib.util.spec_from_file_location("_cola_build", os.path.join(ROOT, "paper_1509_04685_gb300", "build.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    mod.build(checks=True)
    path = str(tmp_path_factory.mktemp("checks") / "checked.npz")
    env = dict(os.environ, COLA_GB300_CHECKS="1", PYTHONPATH=os.pathsep.join([ROOT, TESTS]))
    r = subprocess.run([sys.executable, "-c", f"import test_gpu_checks as t; t.child({path!r})"], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-3000:]
    return dict(np.load(path))


def test_normal_build_has_no_checks():
    assert C.LIB.cola_checks_enabled() == 0
    # in range: runs; out of range: refused on the host (no device check would catch it)
    assert probe() == [(0, 0), (-1, 0), (0, 0), (-1, 0)]


def test_checked_build_latches_a_failed_check(checked):
    # in range: (0, 0); index >= n: launched, the write skipped, COLA_EBOUNDS latched
    assert checked["probe"].tolist() == [[0, 0], [0, -7], [0, 0], [0, -7]]


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("nq,ng,L", CASES)
def test_checked_build_is_bit_identical(checked, nq, ng, L, path):
    ref = outputs(nq, ng, L, path)
    assert int(ref["status"][0]) == 0
    for name in ("status", "force", "d", "v", "density"):
        np.testing.assert_array_equal(checked[f"{nq}_{ng}_{path}_{name}"], ref[name],
                                      err_msg=f"{nq}^3 / {ng}^3 path {path} {name}")
