"""Checkpoint and resume: a run saved after node 19 to a file and resumed in a
fresh Simulation (fresh workspace, cola_init, cola_checkpoint_load) ends
bit-identical to the uninterrupted 40-node run; a checkpoint of one
configuration is refused by another."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import host  # noqa: E402


def test_resumed_run_is_bit_identical(tmp_path):
    cfg = C.make_config(32, 96, 128.0, 0.05)
    full = C.Simulation(cfg)
    full.ic(seed=3)
    full.run()
    part = C.Simulation(cfg)
    part.ic(seed=3)
    part.run(range(20))
    path = str(tmp_path / "run.ckpt")
    part.save_checkpoint(path)
    assert part.node == 20
    del part
    resumed = C.Simulation(cfg)
    resumed.load_checkpoint(path)
    assert resumed.node == 20
    resumed.run(range(20, 40))
    assert resumed.status() == 0
    for name in ("d", "v", "psi1", "psi2"):
        np.testing.assert_array_equal(host(getattr(resumed, name)), host(getattr(full, name)))
    other = C.Simulation(C.make_config(32, 96, 128.0, 0.05, sampling=C.SAMPLING_LOG))
    with pytest.raises(C.ColaError):
        other.load_checkpoint(path)
