"""Training and evaluation of the learned coarse-mesh force correction.

Every arithmetic step runs in the library's kernels (PM forces, least-squares
filter fit, convolution net forward/backward, Adam); this module only
allocates buffers and sequences the calls.

Training data are generated by the method itself: plain COLA runs on a mesh
PM_grid = m_fine times finer than the particle grid (the paper's 3x), whose
states at a few time nodes give particle positions and the fine-mesh force
there.  The correction is then fitted on the PM_grid = 1 mesh:
  1. the radial filter T(|k|) by linear least squares (the gathered force is
     linear in T), and
  2. the convolution net by Adam on L = 1/(2 Np) sum_p |F_1x(p) - F_fine(p)|^2.
"""
from __future__ import annotations

import dataclasses

import numpy as np
import torch

from . import _lib as L
from .sim import Simulation


def init_params(seed: int, device="cuda") -> torch.Tensor:
    """He-scaled first two layers, a small last layer (the correction starts
    near zero), zero biases."""
    g = torch.Generator().manual_seed(seed)
    p = torch.zeros(L.NET_NPARAMS, dtype=torch.float32)
    for k, (off, shape) in L.NET_OFFSETS.items():
        if not k.startswith("W"):
            continue
        n = int(np.prod(shape))
        fan_in = shape[1] * 27
        std = (2.0 / fan_in) ** 0.5 if k != "W3" else 0.01 / fan_in**0.5
        p[off: off + n] = torch.randn(n, generator=g) * std
    return p.to(device)


class LearnedCorrection:
    """Parameters, packed weights, filter table and Adam state of one net."""

    def __init__(self, nfilter: int = 16, seed: int = 0, device="cuda"):
        self.device = torch.device(device)
        self.params = init_params(seed, device)
        self.wpack = torch.zeros(L.NET_NPACK, dtype=torch.bfloat16, device=self.device)
        self.filter = torch.ones(nfilter, dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.net = L.make_net(self.params, self.wpack, self.filter)
        self.pack()

    def pack(self):
        L.cola_net_pack(self.net)

    def config(self, nq: int, box: float, a_init: float = 0.05, n_steps: int = 40, use_net: bool = True):
        """PM_grid = 1 config using this correction (filter always, net if use_net)."""
        if use_net:
            return L.make_config(nq, nq, box, a_init, 1.0, n_steps, flags=L.FLAG_LEARNED, net=self.net)
        zero = LearnedCorrection.__new__(LearnedCorrection)
        zero.params = torch.zeros_like(self.params)
        zero.wpack = torch.zeros_like(self.wpack)
        zero.net = L.make_net(zero.params, zero.wpack, self.filter)
        L.cola_net_pack(zero.net)
        cfg = L.make_config(nq, nq, box, a_init, 1.0, n_steps, flags=L.FLAG_LEARNED, net=zero.net)
        cfg._zero_ref = zero
        return cfg

    def state_dict(self):
        return {"params": self.params.cpu(), "filter": self.filter.cpu()}


@dataclasses.dataclass
class Sample:
    d: torch.Tensor       # (3, Np) displacement of a fine run at node j
    a: float              # scale factor of node j
    force: torch.Tensor   # (3, Np) fine-mesh PM force at those positions


def make_samples(seeds, nq: int, box: float, m_fine: int = 3, nodes=(10, 20, 30, 39), a_init=0.05, n_steps=40,
                 device="cuda"):
    """Run plain COLA at PM_grid = m_fine from each seed and keep (positions,
    fine force) at the given nodes (the force the run itself evaluates there)."""
    out = []
    cfg = L.make_config(nq, m_fine * nq, box, a_init, 1.0, n_steps)
    sim = Simulation(cfg, device=device)
    for seed in seeds:
        sim.ic(seed)
        tab = sim.table()[:, 0].cpu().numpy()
        for j in range(n_steps):
            if j in nodes:
                out.append(Sample(sim.d.clone(), float(tab[j]), sim.force(float(tab[j]))))
            sim.step(j)
    torch.cuda.synchronize()
    return out


def fit_filter(corr: LearnedCorrection, samples, nq: int, box: float, ridge: float = 1e-6):
    """Least-squares radial filter over all samples (normal equations summed)."""
    nb = corr.filter.numel()
    cfg = L.make_config(nq, nq, box, 0.05)
    sim = Simulation(cfg, device=corr.device)
    sim.init_tables()
    basis = torch.empty((nb, 3 * nq**3), dtype=torch.float32, device=corr.device)
    ATA = torch.zeros((nb, nb), dtype=torch.float64, device=corr.device)
    ATy = torch.zeros(nb, dtype=torch.float64, device=corr.device)
    for s in samples:
        sim.d.copy_(s.d)
        L.cola_filter_accumulate(cfg, sim.state, s.a, s.force, nb, basis, ATA, ATy, sim.ws)
    L.cola_filter_solve(ATA, ATy, nb, ridge, corr.filter)
    torch.cuda.synchronize()
    return corr.filter.clone()


def train(corr: LearnedCorrection, samples, nq: int, box: float, iters: int = 500, lr: float = 1e-3, seed: int = 0,
          log_every: int = 0):
    """Adam on the particle loss, one random sample per iteration."""
    cfg = corr.config(nq, box)
    sim = Simulation(cfg, device=corr.device)
    sim.init_tables()
    grad = torch.zeros_like(corr.params)
    loss = torch.zeros(1, dtype=torch.float64, device=corr.device)
    rng = np.random.default_rng(seed)
    hist = []
    for it in range(iters):
        s = samples[rng.integers(len(samples))]
        sim.d.copy_(s.d)
        L.cola_net_grad(cfg, sim.state, s.a, s.force, grad, loss, sim.ws)
        corr.t += 1
        L.cola_adam(corr.params, grad, corr.m, corr.v, L.NET_NPARAMS, corr.t, lr)
        corr.pack()
        if log_every and (it % log_every == 0 or it == iters - 1):
            hist.append((it, float(loss.item())))
    torch.cuda.synchronize()
    return hist


def force_errors(corr: LearnedCorrection, samples, nq: int, box: float):
    """Mean relative L2 force error against the fine force for the plain 1x
    mesh, the 1x mesh with the filter, and the full correction."""
    sims = {
        "plain_1x": Simulation(L.make_config(nq, nq, box, 0.05), device=corr.device),
        "filter_1x": Simulation(corr.config(nq, box, use_net=False), device=corr.device),
        "learned_1x": Simulation(corr.config(nq, box), device=corr.device),
    }
    err = {k: [] for k in sims}
    for s in samples:
        for k, sim in sims.items():
            sim.init_tables()
            sim.d.copy_(s.d)
            f = sim.force(s.a)
            err[k].append(float(torch.linalg.norm(f - s.force) / torch.linalg.norm(s.force)))
    return {k: float(np.mean(v)) for k, v in err.items()}


def run_power(cfg, seed: int, ng_pk: int, device="cuda"):
    """Full 40-step run from the seed's 2LPT field; P(k) at the last node."""
    sim = Simulation(cfg, device=device)
    sim.ic(seed)
    sim.run()
    if sim.status() != 0:
        raise RuntimeError("device status after run")
    k, p, n = sim.power(ng_pk, node=cfg.n_steps - 1)
    return k.cpu().numpy(), p.cpu().numpy()
