"""The N > 1 path of bench.py on CPU: independent replicas, one per rank,
with no data-path collective.  Two gloo ranks check the whole-job reduction
(units of all ranks over the slowest rank's time), the seed and ensemble-member
assignment, and the reference arm under torchrun (rank 0 alone reports)."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _replica_worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # rank r processed 100 (r + 1) units in 10 (r + 1) ms
        value, ms = bench.replica_value(100.0 * (rank + 1), 10.0 * (rank + 1), dist, device="cpu")
        seeds = [0] * world
        dist.all_gather_object(seeds, bench.replica_seed(rank))
        members = [None] * world
        dist.all_gather_object(members, [m[3] for m in bench.members_of(rank, world)])
        out.put((rank, value, ms, seeds, members))
    finally:
        dist.destroy_process_group()


def test_replica_reduction_and_assignment_on_two_gloo_ranks():
    world = 2
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_replica_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = [out.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, value, ms, seeds, members in res:
        assert ms == 20.0                              # the slowest rank's time
        assert value == pytest.approx(300.0 / 20e-3)   # all ranks' units over it
        assert seeds == [1, 2]                         # distinct realisations
        flat = sorted(s for m in members for s in m)
        assert flat == sorted(m[3] for m in bench.ensemble_members())  # every member once


def test_ensemble_members_split_over_any_world_size():
    everyone = sorted(m[3] for m in bench.ensemble_members())
    for world in (1, 2, 3, 4, 8):
        got = sorted(m[3] for r in range(world) for m in bench.members_of(r, world))
        assert got == everyone


def test_reference_arm_under_torchrun_reports_once():
    # the FP64 oracle arm: rank 0 times it and prints one line, rank 1 exits without work
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={_free_port()}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [json.loads(x) for x in r.stdout.splitlines() if x.startswith("{")]
    assert len(lines) == 1
    line = lines[0]
    assert line["impl"] == "reference" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
