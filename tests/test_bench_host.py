"""Host-side logic of bench.py that needs no GPU: the stored ncu traffic is
reported only for the workload and kernel sources it was captured on, and the
algorithmic byte counts follow the stated per-kernel formulas."""
import json
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_stored_traffic_is_keyed_to_workload_and_sources():
    with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
        j = json.load(f)
    w = j["workload"]
    if j["csrc_digest"] == bench.csrc_digest():
        assert bench.ncu_traffic("fft_y_inv", w) == j["kernels"]["fft_y_inv"]["dram_bytes_per_launch_full"]
    assert bench.ncu_traffic("fft_y_inv", w + "_other") is None
    assert bench.ncu_traffic("no_such_kernel", w) is None


def test_traffic_goes_stale_when_a_step_source_changes(tmp_path, monkeypatch):
    # a copy of the tree with one step source edited no longer matches the digest
    csrc = tmp_path / "paper_1509_04685_gb300" / "csrc"
    csrc.mkdir(parents=True)
    for name in bench.STEP_SOURCES:
        src = os.path.join(ROOT, "paper_1509_04685_gb300", "csrc", name)
        (csrc / name).write_bytes(open(src, "rb").read())
    (tmp_path / "profiles").mkdir()
    (tmp_path / "profiles" / "ncu_traffic.json").write_text(
        open(os.path.join(ROOT, "profiles", "ncu_traffic.json")).read())
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.csrc_digest() == bench.csrc_digest()
    before = bench.csrc_digest()
    with open(csrc / bench.STEP_SOURCES[0], "a") as f:
        f.write("\n// edited\n")
    assert bench.csrc_digest() != before
    w = json.loads((tmp_path / "profiles" / "ncu_traffic.json").read_text())["workload"]
    assert bench.ncu_traffic("fft_y_inv", w) is None


@pytest.mark.parametrize("nq,ng", [(512, 1536), (256, 768)])
def test_step_reference_bytes(nq, ng):
    M = 4.0 * ng**3
    Mc = 8.0 * ng * ng * (ng // 2 + 1)
    assert bench.step_reference_bytes(nq, ng) == pytest.approx(M + (M + Mc) + 3 * (Mc + M) + 3 * M + 84.0 * nq**3)
    if (nq, ng) == (512, 1536):
        assert bench.step_reference_bytes(nq, ng) == pytest.approx(185.3e9, rel=1e-3)  # the stated B_ref


def test_algorithmic_bytes_of_the_step_kernels():
    # the per-launch accounting of the kernel table at 512^3 / 1536^3 (GB)
    nq, ng = 512, 1536
    want = {"deposit": 30.60, "fft_z_r2c_fix": 72.50, "fft_y_fwd": 29.03, "fft_x_green": 43.54,
            "fft_y_inv": 72.57, "fft_z_c2r": 87.03, "gather_kick_drift": 53.15,
            # the fused step: bins, deposit + r2c, c2r + gather into 48-byte records, kick + drift
            "bins": 9.16, "dep_r2c": 17.20, "c2r_gather": 52.67, "kick_drift": 16.64}
    for k, gb in want.items():
        assert bench.algorithmic_bytes(k, nq, ng) / 1e9 == pytest.approx(gb, abs=0.01), k
    assert bench.algorithmic_bytes("not_a_kernel", nq, ng) == 0.0
