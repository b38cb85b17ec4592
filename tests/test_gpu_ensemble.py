"""Ensemble of uneven members advanced by one CUDA-graph launch: every member
ends bit-identical to the same member run alone with cola_step (same kernels,
integer deposit), replays are deterministic, and the FFT tile autotuner keeps
results within FFT rounding."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1509_04685_gb300 as C  # noqa: E402

from gpu_util import host, rel_l2  # noqa: E402


def _members():
    out = []
    for i, (nq, m) in enumerate([(16, 1), (16, 2), (16, 3), (24, 1), (24, 2), (32, 3), (20, 2)]):
        cfg = C.make_config(nq, m * nq, float(nq), 0.05, 1.0, 12)
        out.append((cfg, 100 + i))
    return out


def test_graph_ensemble_matches_standalone_runs():
    mem = _members()
    sims = [C.Simulation(cfg) for cfg, _ in mem]
    ens = C.Ensemble([cfg for cfg, _ in mem], [s for _, s in mem], [sm.state for sm in sims], [sm.ws for sm in sims],
                     nstreams=3)
    ens.launch()
    torch.cuda.synchronize()
    first = [host(sm.d).copy() for sm in sims]
    ens.launch()  # replay: ICs + all nodes again
    torch.cuda.synchronize()
    for sm, f in zip(sims, first):
        np.testing.assert_array_equal(host(sm.d), f)
        assert sm.status() == 0
    for (cfg, seed), f in zip(mem, first):
        ref = C.Simulation(cfg)
        ref.ic(seed)
        ref.run()
        np.testing.assert_array_equal(host(ref.d), f)


def test_graph_ensemble_at_the_batched_workload_sizes():
    # the batched workload's member sizes, 40 nodes, L = nq Mpc/h: one member
    # each at 96^3 on 96^3, 128^3 on 256^3 and 160^3 on 480^3 (radices 2, 3, 5)
    mem = [(C.make_config(nq, m * nq, float(nq), 0.05, 1.0, 40), seed)
           for (nq, m), seed in zip([(96, 1), (128, 2), (160, 3)], (1, 17, 33))]
    sims = [C.Simulation(cfg) for cfg, _ in mem]
    ens = C.Ensemble([cfg for cfg, _ in mem], [s for _, s in mem], [sm.state for sm in sims], [sm.ws for sm in sims],
                     nstreams=3)
    ens.launch()
    torch.cuda.synchronize()
    got = [(host(sm.d).copy(), host(sm.v).copy()) for sm in sims]
    for sm in sims:
        assert sm.status() == 0
    del ens, sims
    torch.cuda.empty_cache()
    for (cfg, seed), (d, v) in zip(mem, got):
        ref = C.Simulation(cfg)
        ref.ic(seed)
        ref.run()
        np.testing.assert_array_equal(host(ref.d), d)
        np.testing.assert_array_equal(host(ref.v), v)
        del ref
        torch.cuda.empty_cache()


def test_autotuned_tiles_keep_results():
    n = 96
    cfg = C.make_config(32, n, 128.0, 0.05, 1.0, 6)
    sim = C.Simulation(cfg)
    sim.ic(7)
    sim.run(range(3))
    before = host(sim.force(0.3))
    mesh = torch.zeros(n * n * 2 * C.cola_fft_pitch(n), dtype=torch.float32, device="cuda")
    best = C.cola_fft_autotune(n, mesh, sim.ws)
    assert best in (2, 4, 8, 16)
    after = host(sim.force(0.3))
    assert rel_l2(after, before) < 1e-6
