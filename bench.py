#!/usr/bin/env python
"""Benchmark of the COLA particle-mesh step on GB300.

One "step" is one COLA node (cola_step): CIC deposit, r2c FFT, Green's
function + ik gradient (fused into the x pass), three c2r FFTs, and the fused
CIC gather + kick + drift, on 512^3 particles with a 1536^3 FP32 force mesh
(L = 1536 Mpc/h, 40 linear steps from z = 19; Sec. 2.3 / Table 1 setup with
PM_grid = 3).  The state comes from cola_ic_2lpt (seeded synthetic Gaussian
field); the meshes (14.5 GB each) are far larger than L2, so no flush is
needed between timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload full|small]

Under torchrun each rank advances its own independent realisation (replicas,
seed 1 + rank): the value is the particle-steps of all ranks divided by the
slowest rank's time.  --impl reference times the FP64 CPU oracle on a bounded
sample of the same workload (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "full": dict(name="cola_512^3_particles_1536^3_mesh_L1536_40steps", nq=512, ng=1536, box=1536.0),
    "mid": dict(name="cola_256^3_particles_768^3_mesh_L768_40steps", nq=256, ng=768, box=768.0),
    "largest": dict(name="cola_768^3_particles_2304^3_mesh_L1536_40steps", nq=768, ng=2304, box=1536.0),
    "small": dict(name="cola_32^3_particles_96^3_mesh_L128_40steps", nq=32, ng=96, box=128.0),
    # 48 seeds: 16 each at 96^3, 128^3, 160^3 particles, PM_grid cycling 1, 2, 3, L = 1 Mpc/h per spacing
    "ensemble": dict(name="cola_ensemble_48_seeds_96-128-160^3_pm1-2-3_40steps", nq=0, ng=0, box=0.0),
    # learned 1x mesh vs plain 3x mesh, 256^3 particles, L = 512 Mpc/h
    "learned": dict(name="cola_learned_256^3_particles_256^3_vs_768^3_mesh_L512_40steps", nq=0, ng=0, box=0.0),
    # the largest run's learned 1.5x form vs its plain 3x form, P(k) at z = 1, 0.5, 0
    "largest_learned": dict(name="cola_learned_768^3_particles_1152^3_vs_2304^3_mesh_L1536_40steps", nq=0, ng=0,
                            box=0.0),
    # convergence in the number of time steps (10/20/40 against 80), every time sampling
    # and both kick/drift forms, at 32^3/96^3 (L = 128) and 256^3/768^3 (L = 768)
    "convergence": dict(name="cola_convergence_10-20-40_vs_80_steps_32^3_96^3_and_256^3_768^3", nq=0, ng=0, box=0.0),
}


def max_over_ranks(x: float, dist, device="cuda") -> float:
    """The slowest rank's value (every rank receives it); x itself without a process group."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, dist, device="cuda") -> float:
    """The sum over ranks (every rank receives it); x itself without a process group."""
    if not dist:
        return x
    import torch

    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


def replica_value(units_local: float, ms_local: float, dist, device="cuda") -> tuple[float, float]:
    """Whole-job throughput of independent replicas: the units of all ranks
    over the slowest rank's time.  Returns (value per second, max ms)."""
    ms = max_over_ranks(ms_local, dist, device)
    return sum_over_ranks(units_local, dist, device) / (ms * 1e-3), ms


def replica_seed(rank: int) -> int:
    """Realisation of a rank: seed 1 + rank (rank 0 runs the single-GPU seed)."""
    return 1 + rank


def members_of(rank: int, world: int):
    """The ensemble members a rank advances: member i on rank i mod world."""
    return [m for i, m in enumerate(ensemble_members()) if i % world == rank]


def ensemble_members():
    out = []
    for i in range(48):
        nq = (96, 128, 160)[i // 16]
        m = 1 + i % 3
        out.append((nq, m * nq, float(nq), 1 + i))
    return out


def run_ensemble(args, rank, world, C, torch, dist):
    """One timed step = one graph launch replaying the 2LPT set-up and all 40
    nodes of this rank's members (members i = rank mod world)."""
    line = ensemble_line(C, torch, dist, rank, world, max(1, args.warmup // 3), max(1, args.steps // 12))
    if rank == 0:
        print(json.dumps(line), flush=True)


def ensemble_line(C, torch, dist, rank, world, warmup, nrep):
    """The ensemble's JSON line (see run_ensemble)."""
    mem = members_of(rank, world)
    cfgs = [C.make_config(nq, ng, box, A_INIT, 1.0, N_NODES) for nq, ng, box, _ in mem]
    sims = [C.Simulation(c) for c in cfgs]
    # autotune the tile width of every mesh size once
    scratch_n = max(c.ng for c in cfgs)
    scratch = torch.zeros(scratch_n * scratch_n * 2 * C.cola_fft_pitch(scratch_n), dtype=torch.float32,
                          device="cuda")
    tuned = {}
    for c, sm in zip(cfgs, sims):
        for n in (c.ng, c.nq):
            if n not in tuned:
                tuned[n] = C.cola_fft_autotune(n, scratch, sm.ws)
    del scratch
    # one uncaptured step per member sets kernel attributes before capture
    for c, sm, (_, _, _, seed) in zip(cfgs, sims, mem):
        sm.ic(seed)
        sm.step(0)
    ens = C.Ensemble(cfgs, [m[3] for m in mem], [sm.state for sm in sims], [sm.ws for sm in sims], nstreams=8)
    for _ in range(warmup):
        ens.launch()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    launches0 = C.cola_launch_count()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(nrep):
        ens.launch()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    for sm in sims:
        if sm.status() != 0:
            raise SystemExit("device status after ensemble")
    value, ms = replica_value(float(sum(nq**3 for nq, _, _, _ in mem) * N_NODES * nrep), ms, dist)
    launches = C.cola_launch_count() - launches0
    del ens, sims
    torch.cuda.empty_cache()
    return {
        "metric": "particle-steps/s (48-seed uneven ensemble, one CUDA-graph launch per run)", "value": value,
        "unit": UNIT, "n_gpus": world, "steps": nrep, "warmup": warmup,
        "ms_per_step": ms / nrep, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOADS["ensemble"]["name"], "members": 48, "n_steps": N_NODES,
                   "step": "one graph launch = 2LPT set-up + 40 nodes of every member",
                   "autotuned_tiles": {str(k): v for k, v in sorted(tuned.items())},
                   "parallelism": f"members sharded over {world} rank(s)"},
        "clocks": clk, "gpu_launches": launches,
    }
def learned_study(C, torch, nq, box, train_seeds, test_seeds, net_iters, dev_index=0):
    """The learned 1x-mesh form against the plain 3x-mesh form (config 4 at
    nq = 256, L = 512 Mpc/h, 40 steps).  The radial filter is fitted by least
    squares on every node of plain 3x runs of the training seeds and its
    P(k) calibration on four of them; the learned form is the filtered 1x mesh
    alone.  With net_iters > 0 the convolution net is also trained (on four
    nodes of the first eight runs) and reported as a separate form.  Every form
    then runs the held-out seeds; returns the timings and the final P(k)
    deviation from the plain 3x form for k <= 1 h/Mpc."""
    import numpy as np

    from paper_1509_04685_gb300 import learn

    t0 = time.perf_counter()
    corr = learn.LearnedCorrection(nfilter=16, seed=0, nfilter_a=8)
    samples, final = learn.fit_filter_runs(corr, train_seeds, nq, box,
                                           keep_nodes=(10, 20, 30, 39) if net_iters else ())
    hist = []
    if net_iters:
        hist = learn.train(corr, samples[: 4 * 8], nq, box, iters=net_iters, lr=3e-3,
                           log_every=max(1, net_iters // 4))
    del samples
    torch.cuda.empty_cache()
    cal = {s: final[s] for s in train_seeds[:4]}
    gain, boost = learn.calibrate_filter(corr, cal, nq, box, use_net=False)
    t_train = time.perf_counter() - t0
    forms = {"plain_3x": C.make_config(nq, 3 * nq, box, A_INIT, 1.0, N_NODES),
             "plain_1x": C.make_config(nq, nq, box, A_INIT, 1.0, N_NODES),
             "learned_1x": corr.config(nq, box, use_net=False)}
    if net_iters:
        forms["learned_1x_net"] = corr.config(nq, box, use_net=True)
    sims = {k: C.Simulation(cfg) for k, cfg in forms.items()}
    ms = {k: 0.0 for k in sims}
    pk = {k: [] for k in sims}
    clocks = Clocks(dev_index)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for key, sm in sims.items():  # one untimed run per form (kernel attributes, caches)
        sm.ic(test_seeds[0])
        sm.run()
    for seed in test_seeds:
        for key, sm in sims.items():
            sm.ic(seed)
            torch.cuda.synchronize()
            e0.record()
            sm.run()
            e1.record()
            torch.cuda.synchronize()
            ms[key] += e0.elapsed_time(e1)
            if sm.status() != 0:
                raise SystemExit(f"device status after the {key} run")
            k, p, _ = sm.power(nq, node=N_NODES - 1)
            pk[key].append(p.cpu().numpy())
    clk = clocks.stop()
    k = k.cpu().numpy()
    sel = k <= 1.0
    ratio = {key: np.mean(np.stack(pk[key]), axis=0) / np.mean(np.stack(pk["plain_3x"]), axis=0) for key in pk}
    others = [key for key in sims if key != "plain_3x"]
    dev = {key: float(np.max(np.abs(ratio[key][sel] - 1))) for key in others}
    mdev = {key: float(np.mean(np.abs(ratio[key][(k > 0.1) & sel] - 1))) for key in others}
    nsteps = N_NODES * len(test_seeds)
    del sims
    torch.cuda.empty_cache()
    return {
        "ms_per_step": {key: ms[key] / nsteps for key in ms},
        "particle_steps_per_s": {key: nq**3 * nsteps / (ms[key] * 1e-3) for key in ms},
        "speedup_vs_plain_3x": ms["plain_3x"] / ms["learned_1x"],
        "pk_final": {"k_max": 1.0, "target_max_abs_dev": 0.01, "max_abs_dev": dev, "mean_abs_dev_0.1_to_1": mdev,
                     "learned_within_target": dev["learned_1x"] <= 0.01,
                     "ratio_learned": [round(float(x), 5) for x in ratio["learned_1x"][sel]],
                     "ratio_plain_1x": [round(float(x), 5) for x in ratio["plain_1x"][sel]],
                     "k": [round(float(x), 4) for x in k[sel]]},
        "training": {"seconds": t_train, "train_seeds": len(train_seeds), "test_seeds": len(test_seeds),
                     "net_iters": net_iters, "net_loss": hist, "filter_gain": gain, "filter_boost": boost,
                     "calibration_seeds": len(cal)},
        "clocks": clk, "steps": nsteps,
    }


def run_learned(args, rank, world, C, torch, dist):
    """Config 4: the learned 1x-mesh form (the filtered coarse mesh) against the
    plain 3x-mesh form, 256^3 particles, L = 512 Mpc/h; the value is the learned
    form's particle-steps/s (summed over replicas)."""
    nq, box = 256, 512.0
    train_seeds = [1001 + 100 * rank + i for i in range(args.learned_train)]
    test_seeds = [2001 + 100 * rank + i for i in range(args.learned_test)]
    launches0 = C.cola_launch_count()
    st = learned_study(C, torch, nq, box, train_seeds, test_seeds, args.learned_iters,
                       int(os.environ.get("LOCAL_RANK", "0")))
    ps = st["particle_steps_per_s"]
    tot = torch.tensor([ps["learned_1x"], ps["plain_3x"]], device="cuda")
    if dist:
        dist.all_reduce(tot)
    if rank == 0:
        print(json.dumps({
            "metric": "particle-steps/s of the learned 1x-mesh form (256^3 particles, L=512 Mpc/h)",
            "value": float(tot[0].item()), "unit": UNIT, "n_gpus": world, "steps": st["steps"], "warmup": N_NODES,
            "ms_per_step": st["ms_per_step"]["learned_1x"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["learned"]["name"], "nq": nq, "ng_learned": nq, "ng_plain": 3 * nq,
                       "box": box, "n_steps": N_NODES, "train_seeds": len(train_seeds), "test_seeds": len(test_seeds),
                       "learned_form": "radial filter on the 1x mesh (16 nodes x 8 scale-factor rows, least squares "
                                       "on every node of the fine runs, P(k)-calibrated boost); the convolution net "
                                       "is reported apart as learned_1x_net when trained (--learned-iters)",
                       "parallelism": f"replicas{world}"},
            "plain_3x": {"value": float(tot[1].item()), "ms_per_step": st["ms_per_step"]["plain_3x"]},
            "forms": st["ms_per_step"], "speedup_vs_plain_3x": st["speedup_vs_plain_3x"],
            "pk_final": st["pk_final"], "training": st["training"], "clocks": st["clocks"],
            "gpu_launches": C.cola_launch_count() - launches0,
        }), flush=True)


def run_convergence(args, rank, world, C, torch, dist):
    """Convergence of the final P(k) in the number of time steps, in the spirit
    of the paper's Sec. 4.1-4.3 study (there against MICE-GC, here internal):
    runs of 10, 20 and 40 steps from z = 19, with the linear, log and a^0.5
    samplings of Eq. 3 and with the standard or the Tassev et al. (2013) kick
    and drift factors, against 80 linear steps with the standard factors from
    the same seed.  Reported per run: max |P/P_80 - 1| for k <= 0.5 and k <= 1
    h/Mpc (P(k) on the force mesh, final node), and the run's ms per step."""
    import numpy as np

    if rank != 0:
        return
    cases = [(32, 96, 128.0), (256, 768, 768.0)]
    samplings = (("linear", C.SAMPLING_LINEAR, 1.0), ("log", C.SAMPLING_LOG, 1.0), ("a^0.5", C.SAMPLING_POW, 0.5))
    out = {}
    launches0 = C.cola_launch_count()
    for nq, ng, box in cases:
        def final_pk(n, sampling=C.SAMPLING_LINEAR, p=1.0, flags=0):
            sim = C.Simulation(C.make_config(nq, ng, box, A_INIT, 1.0, n, sampling=sampling, sampling_p=p,
                                             flags=flags))
            sim.ic(seed=1)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            sim.run()
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / n
            if sim.status() != 0:
                raise SystemExit(f"device status after the {n}-step run")
            k, pk, _ = sim.power(ng, node=n - 1)
            res = (k.cpu().numpy(), pk.cpu().numpy(), ms)
            del sim
            torch.cuda.empty_cache()
            return res

        k, p80, _ = final_pk(80)
        rows = []
        for kdk, flags in (("standard", 0), ("modified", C.FLAG_MODIFIED_KDK)):
            for sname, samp, sp in samplings:
                for n in (10, 20, 40):
                    _, pn, ms = final_pk(n, samp, sp, flags)
                    r = pn / p80 - 1
                    rows.append({"steps": n, "sampling": sname, "kdk": kdk,
                                 "max_dev_k<=0.5": float(np.max(np.abs(r[k <= 0.5]))),
                                 "max_dev_k<=1": float(np.max(np.abs(r[k <= 1.0]))),
                                 "ms_per_step": round(ms, 3)})
        out[f"{nq}^3_{ng}^3_L{box:g}"] = {"k_nyquist": float(np.pi * ng / box), "runs": rows}
    print(json.dumps({
        "metric": "final P(k) deviation from 80 linear steps", "unit": "max |P/P_80 - 1|", "n_gpus": 1,
        "higher_is_better": False, "data": "synthetic", "dtype": "f32",
        "config": {"workload": WORKLOADS["convergence"]["name"], "z_init": 1 / A_INIT - 1, "seed": 1},
        "results": out, "gpu_launches": C.cola_launch_count() - launches0,
    }), flush=True)


def run_largest_learned(args, rank, world, C, torch, dist):
    """The largest run's two forms at the same seed: plain PM_grid = 3 (768^3
    particles on 2304^3) and the learned 1.5x form (768^3 on 1152^3), L = 1536
    Mpc/h, 40 steps, P(k) at z = 1, 0.5 and 0 on a 768^3 mesh.  The learned form
    is the radial filter alone: the net's activations would need ~150 GB at
    1152^3.  The filter is fitted and calibrated in a 128^3 / L = 256 box at the
    same resolution (its nodes are fixed in k L / ng).  The value is the learned
    form's particle-steps/s."""
    import numpy as np

    from paper_1509_04685_gb300 import learn

    t0 = time.perf_counter()
    nq_t, box_t = 128, 256.0
    train_seeds = [1001 + 100 * rank + i for i in range(args.learned_train)]
    corr = learn.LearnedCorrection(nfilter=16, seed=0, nfilter_a=8, mesh_factor=1.5)
    _, final = learn.fit_filter_runs(corr, train_seeds, nq_t, box_t, outputs=(0.5, 2.0 / 3.0, 1.0))
    gain, boost = learn.calibrate_filter(corr, {s: final[s] for s in train_seeds[:4]}, nq_t, box_t, use_net=False)
    torch.cuda.empty_cache()
    t_train = time.perf_counter() - t0

    nq, box, ng_pk, seed = 768, 1536.0, 768, 1 + rank
    a_nodes = A_INIT + np.arange(N_NODES) * (1.0 - A_INIT) / (N_NODES - 1)
    outputs = [(1.0, 0.5), (0.5, 2.0 / 3.0), (0.0, 1.0)]  # (z, a)
    clocks = Clocks(int(os.environ.get("LOCAL_RANK", "0")))
    launches0 = C.cola_launch_count()

    def run(cfg):
        sim = C.Simulation(cfg)
        sim.ic(seed)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ms, pks, j = 0.0, {}, 0
        for z, a in outputs:
            node = N_NODES - 1 if a >= 1.0 else int(np.floor((a - A_INIT) / (a_nodes[1] - a_nodes[0]) + 1e-9))
            torch.cuda.synchronize()
            e0.record()
            sim.run(range(j, node if a < 1.0 else N_NODES))
            e1.record()
            torch.cuda.synchronize()
            ms += e0.elapsed_time(e1)
            j = node if a < 1.0 else N_NODES
            k, p, _ = sim.power(ng_pk, a_out=a, node=node)
            pks[z] = (k.cpu().numpy(), p.cpu().numpy())
        if sim.status() != 0:
            raise SystemExit("device status after the largest run")
        del sim
        torch.cuda.empty_cache()
        return ms, pks

    ms3, pk3 = run(C.make_config(nq, 3 * nq, box, A_INIT, 1.0, N_NODES))
    msl, pkl = run(corr.config(nq, box, use_net=False))
    clk = clocks.stop()
    pkdev = {}
    for z, _ in outputs:
        k, p3 = pk3[z]
        _, pl = pkl[z]
        sel = k <= 1.0
        pkdev[f"z={z:g}"] = {"max_abs_dev": float(np.max(np.abs(pl[sel] / p3[sel] - 1))),
                             "mean_abs_dev": float(np.mean(np.abs(pl[sel] / p3[sel] - 1))),
                             "ratio_at_k": {f"{kk:.2f}": round(float(r), 4) for kk, r in
                                            zip(k[sel][::10], (pl[sel] / p3[sel])[::10])}}
    ps_l = nq**3 * N_NODES / (msl * 1e-3)
    ps_3 = nq**3 * N_NODES / (ms3 * 1e-3)
    tot = torch.tensor([ps_l, ps_3], device="cuda")
    if dist:
        dist.all_reduce(tot)
    if rank == 0:
        print(json.dumps({
            "metric": "particle-steps/s of the learned 1.5x-mesh form (768^3 particles on 1152^3, L=1536 Mpc/h)",
            "value": float(tot[0].item()), "unit": UNIT, "n_gpus": world, "steps": N_NODES, "warmup": 0,
            "ms_per_step": msl / N_NODES, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOADS["largest_learned"]["name"], "nq": nq, "ng_learned": 1152,
                       "ng_plain": 3 * nq, "box": box, "n_steps": N_NODES, "seed": seed,
                       "correction": "radial filter alone (16 k nodes x 8 scale-factor rows), fitted on "
                                     f"{len(train_seeds)} runs of 128^3 on 192^3 vs 384^3 (L=256), calibrated on 4 "
                                     "at z = 1, 0.5, 0",
                       "pk_mesh": ng_pk, "parallelism": f"replicas{world}"},
            "plain_3x": {"value": float(tot[1].item()), "ms_per_step": ms3 / N_NODES},
            "speedup_vs_plain_3x": ps_l / ps_3,
            "pk_vs_plain_3x_k_le_1": pkdev,
            "training": {"seconds": t_train, "filter_gain": gain, "filter_boost": boost},
            "clocks": clk, "gpu_launches": C.cola_launch_count() - launches0,
        }), flush=True)


A_INIT, N_NODES = 0.05, 40
METRIC = "particle-steps/s at 512^3/1536^3"
METRICS = {"largest": "particle-steps/s at 768^3/2304^3", "mid": "particle-steps/s at 256^3/768^3",
           "small": "particle-steps/s at 32^3/96^3"}
UNIT = "particle-steps/s"
FALLBACK_HBM = 6800.0


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            j = json.load(f)
        return float(j["hbm_gbs"]), "measured"
    return FALLBACK_HBM, "fallback"


def algorithmic_bytes(name: str, nq: int, ng: int) -> float:
    """Bytes each kernel must move per launch (one HBM read of its inputs and
    one write of its outputs; FP32 mesh values, 8-byte fixed-point counts)."""
    Np = nq**3
    Mc = ng * ng * (ng // 2 + 1) * 8.0  # half-complex mesh
    M = ng**3 * 4.0                     # real mesh
    F = ng**3 * 8.0                     # fixed-point CIC mesh
    return {
        # row bins: positions read, key + rank written (count); key, rank, positions and
        # the bin offset read, index, CIC record and sorted position written (scatter);
        # the ng^2 counts cleared, counted, scanned (read + write) and read
        "bins": 68.0 * Np + 16.0 * ng * ng,
        # each particle's CIC record and index read once, delta_k written
        "dep_r2c": 20.0 * Np + Mc,
        # three force components read, CIC records and indices read once, the
        # 48-byte partial-sum records written
        "c2r_gather": 3 * Mc + 20.0 * Np + 48.0 * Np,
        # sorted position and partial-sum record, d, v, psi1, psi2 read; d, v written
        "kick_drift": 52.0 * Np + 72.0 * Np,
        "deposit": 12.0 * Np + F,
        "fft_z_r2c_fix": 2 * F + Mc,
        "fft_y_fwd": 2 * Mc, "fft_x_fwd": 2 * Mc, "fft_x_inv": 2 * Mc,
        # the fused x pass writes F_x and Psi = IFFT_x(phi); the y inverse reads both and
        # writes F_x, F_y = IFFT_y(i k_y Psi) and F_z = i k_z IFFT_y(Psi)
        "fft_y_inv": 5 * Mc,
        "fft_x_green": 3 * Mc,
        "fft_z_c2r": 3 * (Mc + M),    # all three force components in one launch
        "gather_kick_drift": 72.0 * Np + 3 * M,
    }.get(name, 0.0)


def step_reference_bytes(nq: int, ng: int) -> float:
    """B_ref per PM step: density written, one read+write per 3D transform,
    the three force meshes read once, 84 bytes per particle."""
    M = ng**3 * 4.0
    Mc = ng * ng * (ng // 2 + 1) * 8.0
    return M + (M + Mc) + 3 * (Mc + M) + 3 * M + 84.0 * nq**3


# sources that define and launch the kernels of a step (profiles/ncu_traffic.json
# holds counters taken on them; a change here makes the stored traffic stale)
STEP_SOURCES = ("cola_common.cuh", "fft_static.cuh", "fft_fused.cuh", "particles.cuh", "fft.cu", "fft_spec_large.cu",
                "fft_spec_small.cu", "pm.cu", "scan.cu", "api.cu")


def csrc_digest() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_1509_04685_gb300", "csrc")
    for f in STEP_SOURCES:
        with open(os.path.join(d, f), "rb") as fh:
            h.update(f.encode() + fh.read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources and on this workload (else None)."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    with open(p) as f:
        j = json.load(f)
    if j.get("csrc_digest") != csrc_digest() or j.get("workload") != workload:
        return None
    k = j.get("kernels", {}).get(kernel)
    return None if k is None else float(k["dram_bytes_per_launch_full"])


class Clocks:
    """nvidia-smi sampler (200 ms) running across the timed region."""

    def __init__(self, dev_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(dev_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def host_cpu():
    """(threads, model) of the host: all cores serve the oracle's FFTs."""
    n = os.cpu_count() or 1
    model = platform.machine()
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return n, model


def oracle_threads():
    """Give the oracle's FFTs (scipy.fft pocketfft) every host core; returns
    the thread count and a description for the baseline's sample string."""
    from oracle import lpt

    n, model = host_cpu()
    lpt.FFT_WORKERS = n
    return n, (f"{n} host threads ({model}): FFTs on scipy.fft with workers={n}, "
               "the CIC deposit/gather (np.bincount) and elementwise NumPy single-threaded")


def cpu_baseline(nq=128, ng=384, box=384.0):
    """The FP64 oracle (as it stands) for one PM step on a bounded sample of the
    workload: same particle spacing (3 Mpc/h) and PM_grid = 3, 128^3 particles."""
    import numpy as np

    from oracle import cola as ocola
    from oracle import cosmology as cm
    from oracle import lpt

    cores, how = oracle_threads()
    c = cm.Cosmology()
    g = cm.Growth(c)
    tab = cm.step_table(c, cm.time_nodes(A_INIT, 1.0, N_NODES), g)
    st = lpt.initial_conditions(1, nq, box, cm.LinearPower(c), tab.D1[0], tab.D2[0])
    t0 = time.perf_counter()
    ocola.cola_step(st, 20, tab, nq, ng, box)
    dt = time.perf_counter() - t0
    return {"value": nq**3 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"one PM step (node 20) of the FP64 NumPy oracle at {nq}^3 particles on a {ng}^3 mesh, "
                      f"L={box:g} Mpc/h (same spacing and PM_grid as the workload), {dt:.1f} s; {how}"}


def run_reference(args, rank):
    if rank != 0:
        return
    import numpy as np

    from oracle import cola as ocola
    from oracle import cosmology as cm
    from oracle import lpt

    nq, ng, box = 64, 192, 192.0
    cores, how = oracle_threads()
    c = cm.Cosmology()
    tab = cm.step_table(c, cm.time_nodes(A_INIT, 1.0, N_NODES), cm.Growth(c))
    st = lpt.initial_conditions(1, nq, box, cm.LinearPower(c), tab.D1[0], tab.D2[0])
    for j in range(args.warmup):
        ocola.cola_step(st, j % N_NODES, tab, nq, ng, box)
    t0 = time.perf_counter()
    for i in range(args.steps):
        ocola.cola_step(st, (args.warmup + i) % N_NODES, tab, nq, ng, box)
    dt = time.perf_counter() - t0
    value = nq**3 * args.steps / dt
    sample = (f"FP64 NumPy oracle, {nq}^3 particles on a {ng}^3 mesh, L={box:g} Mpc/h (same spacing and "
              f"PM_grid as the workload); {how}")
    w = WORKLOADS[args.workload]
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": w["name"], "nq": w["nq"], "ng": w["ng"], "box": w["box"], "n_steps": N_NODES,
                   "sample_nq": nq, "sample_ng": ng},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=37)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="full", choices=list(WORKLOADS))
    ap.add_argument("--e2e-steps", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--learned-train", type=int, default=32, help="fine training runs (learned workload)")
    ap.add_argument("--learned-test", type=int, default=8, help="held-out seeds (learned workload)")
    ap.add_argument("--learned-iters", type=int, default=0,
                    help="Adam iterations of the convolution net (learned workload; 0: the filter alone)")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-form summary of the default line")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ensemble summary of the default line")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank)
        return

    import torch

    import paper_1509_04685_gb300 as C

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    if args.workload in ("ensemble", "learned", "largest_learned", "convergence"):
        {"ensemble": run_ensemble, "learned": run_learned, "largest_learned": run_largest_learned,
         "convergence": run_convergence}[args.workload](args, rank, world, C, torch, dist)
        if dist:
            dist.destroy_process_group()
        return
    w = WORKLOADS[args.workload]
    cfg = C.make_config(w["nq"], w["ng"], w["box"], A_INIT, 1.0, N_NODES)
    import ctypes
    pm_path = {1: "fused", 2: "separate"}.get(C.LIB.cola_pm_path(ctypes.byref(cfg)), "unknown")
    sim = C.Simulation(cfg, device=f"cuda:{local}")
    sim.ic(seed=replica_seed(rank))
    for j in range(args.warmup):
        sim.step(j % N_NODES)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = Clocks(local)
    time.sleep(0.3)
    nk = C.LIB.cola_num_kernel_ids()
    launches0 = C.cola_launch_count()
    C.LIB.cola_profile_start(args.steps * 16 + 64)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for i in range(args.steps):
        sim.step((args.warmup + i) % N_NODES)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    launches = C.cola_launch_count() - launches0
    kms = (ctypes.c_double * nk)()
    kcnt = (ctypes.c_int64 * nk)()
    C.LIB.cola_profile_stop(kms, kcnt, nk)
    clk = clocks.stop()
    status = sim.status()
    if status != 0:
        raise SystemExit(f"device status {status}: {C.cola_strerror(status)}")
    value, ms = replica_value(float(w["nq"] ** 3 * args.steps), ms, dist)
    if dist:
        dist.barrier()

    per_kernel = {}
    for i in range(nk):
        if kcnt[i]:
            name = C.LIB.cola_kernel_name(i).decode()
            per_kernel[name] = {"launches": int(kcnt[i]), "ms": kms[i], "share": kms[i] / max(ms, 1e-9)}
    dom = max(per_kernel, key=lambda k: per_kernel[k]["ms"])
    dom_avg_ms = per_kernel[dom]["ms"] / per_kernel[dom]["launches"]
    alg = algorithmic_bytes(dom, w["nq"], w["ng"])
    peak, peak_kind = peaks()
    achieved = alg / (dom_avg_ms * 1e-3) / 1e9
    np_total = w["nq"] ** 3 * world
    step_ms = ms / args.steps
    bref = step_reference_bytes(w["nq"], w["ng"])

    # the outputs' cost, timed apart from the step: P(k) and the redshift-space
    # multipoles of the current state on a 1024^3 estimator mesh (the paper's P(k)
    # mesh), and the FoF halos (b = 0.2, more than 100 particles) with their catalogue
    pk_ms = {}
    ng_pk = min(1024, w["ng"])
    fof_out = {}

    def run_fof():
        fof_out["halos"] = int(sim.fof(0.2, 101)[1].numel())

    for name, call in (("power_spectrum", lambda: sim.power(ng_pk)), ("multipoles", lambda: sim.multipoles(ng_pk)),
                       ("power_spectrum_jing_iterated", lambda: sim.power(ng_pk, flags=C.PK_ALIAS_ITER)),
                       ("fof_halos", run_fof)):
        call()
        torch.cuda.synchronize()
        e4, e5 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e4.record()
        call()
        e5.record()
        torch.cuda.synchronize()
        pk_ms[name] = e4.elapsed_time(e5)

    # end to end through the C ABI with host buffers (cola_step_host): per step
    # the state (d, v, psi1, psi2) goes in from pinned host memory and (d, v)
    # come back into it before the call returns
    ke = max(1, args.e2e_steps)
    hst = [torch.empty_like(x, device="cpu").pin_memory() for x in (sim.d, sim.v, sim.psi1, sim.psi2)]
    for h, x in zip(hst, (sim.d, sim.v, sim.psi1, sim.psi2)):
        h.copy_(x)
    host_state = C.make_state(*hst)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record()
    for i in range(ke):
        sim.step_host(host_state, (args.warmup + args.steps + i) % N_NODES)
    e3.record()
    torch.cuda.synchronize()
    ms_e2e = max_over_ranks(e2.elapsed_time(e3), dist)
    h2d = sum(x.numel() * x.element_size() for x in hst)
    d2h = sum(x.numel() * x.element_size() for x in hst[:2])

    # config 4 alongside the headline: the learned 1x-mesh form against the plain
    # 3x form (filter fitted on 8 training seeds, 4 held-out seeds), so that its
    # speed and its P(k) deviation for k <= 1 h/Mpc are on the default line too
    learned = None
    if rank == 0 and args.workload == "full" and not args.no_learned:
        del sim, hst, host_state
        torch.cuda.empty_cache()
        try:
            st = learned_study(C, torch, 256, 512.0, [1001 + i for i in range(8)], [2001 + i for i in range(4)], 0,
                               local)
            learned = {"workload": WORKLOADS["learned"]["name"], "ms_per_step": st["ms_per_step"],
                       "particle_steps_per_s": st["particle_steps_per_s"],
                       "speedup_vs_plain_3x": st["speedup_vs_plain_3x"],
                       "pk_final_max_abs_dev_k<=1": st["pk_final"]["max_abs_dev"],
                       "pk_final_mean_abs_dev_0.1<k<=1": st["pk_final"]["mean_abs_dev_0.1_to_1"],
                       "within_1pct": st["pk_final"]["learned_within_target"],
                       "train_seeds": 8, "test_seeds": 4, "training_s": st["training"]["seconds"]}
        except Exception as e:  # the headline stands without it
            learned = {"error": f"{type(e).__name__}: {e}"}
    # config 3 alongside the headline at N = 1: one run of the 48-member ensemble
    # (one graph launch; its own warm-up launch first)
    ensemble = None
    if world == 1 and args.workload == "full" and not args.no_ensemble:
        if learned is None:
            del sim, hst, host_state
        torch.cuda.empty_cache()
        try:
            e = ensemble_line(C, torch, None, 0, 1, 1, 1)
            ensemble = {"workload": e["config"]["workload"], "value": e["value"], "unit": e["unit"],
                        "ms_per_run": e["ms_per_step"], "runs": e["steps"], "members": 48, "n_steps": N_NODES,
                        "clocks": e["clocks"], "gpu_launches": e["gpu_launches"]}
        except Exception as e:  # the headline stands without it
            ensemble = {"error": f"{type(e).__name__}: {e}"}
    if rank == 0:
        cpu = None if args.no_cpu_baseline else cpu_baseline()
        line = {
            "metric": METRICS.get(args.workload, METRIC), "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": w["name"], "nq": w["nq"], "ng": w["ng"], "box": w["box"], "n_steps": N_NODES,
                       "z_init": 1 / A_INIT - 1, "parallelism": f"replicas{world}", "pm_path": pm_path,
                       "l2": "inputs larger than L2 (every mesh >> 129 MB); no flush"},
            "clocks": clk,
            "gpu_launches": launches,
            "e2e": {"value": np_total * ke / (ms_e2e * 1e-3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": ke},
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "peak_kind": f"of {peak_kind}",
                         "algorithmic_bytes_per_launch": alg, "traffic": ncu_traffic(dom, w["name"])},
            "step_roofline": {"B_ref_bytes": bref, "achieved_GBs": bref / (step_ms * 1e-3) / 1e9,
                              "frac": bref / (step_ms * 1e-3) / 1e9 / peak},
            "kernels": per_kernel,
            "outputs_ms": {"ng_pk": ng_pk, **pk_ms, "fof_n_halos": fof_out.get("halos"),
                           "fof_after_nodes": args.warmup + args.steps},
            "cpu_baseline": cpu,
        }
        if learned is not None:
            line["learned_1x"] = learned
        if ensemble is not None:
            line["ensemble"] = ensemble
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
