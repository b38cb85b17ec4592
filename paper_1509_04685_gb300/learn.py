"""Training and evaluation of the learned coarse-mesh force correction.

Every arithmetic step on particles and meshes runs in the library's kernels
(PM forces, least-squares filter fit, convolution net forward/backward, Adam);
this module allocates buffers and sequences the calls.  The one exception is
the calibration of the fitted filter (calibrated_filter): a reshaping of its
table of nfilter_a x nfilter values by two scalars, done with torch between
training runs.  It is part of training, not of the PM step.

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


def filter_row(a: float, nrows: int, a_init: float = 0.05, a_final: float = 1.0) -> int:
    """Row of a scale-factor-dependent filter table used at scale factor a:
    the nearest of nrows nodes spaced linearly from a_init to a_final."""
    if nrows <= 1:
        return 0
    u = (a - a_init) / (a_final - a_init) * (nrows - 1)
    return int(min(max(np.floor(u + 0.5), 0), nrows - 1))


class LearnedCorrection:
    """Parameters, packed weights, filter table and Adam state of one net.
    The radial filter has nfilter_a rows, one per scale-factor node.  The
    coarse mesh has mesh_factor cells per particle spacing (1 for the paper's
    PM_grid = 1, 1.5 for the largest run's learned form); the filter nodes are
    fixed in k L / ng, so a correction fitted in a small box applies to a
    larger one at the same resolution."""

    def __init__(self, nfilter: int = 16, seed: int = 0, device="cuda", nfilter_a: int = 1, mesh_factor: float = 1.0):
        self.device = torch.device(device)
        self.mesh_factor = mesh_factor
        self.params = init_params(seed, device)
        self.wpack = torch.zeros(L.NET_NPACK, dtype=torch.bfloat16, device=self.device)
        self.filter = torch.ones((nfilter_a, nfilter), dtype=torch.float32, device=self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.t = 0
        self.net = L.make_net(self.params, self.wpack, self.filter)
        self.pack()

    def pack(self):
        L.cola_net_pack(self.net)

    def ng(self, nq: int) -> int:
        """Coarse mesh cells per side for nq particles per side."""
        return int(round(self.mesh_factor * nq))

    def config(self, nq: int, box: float, a_init: float = 0.05, n_steps: int = 40, use_net: bool = True):
        """Coarse-mesh config using this correction: the filter always, the net
        if use_net (else the filter alone: no net buffers, no convolutions)."""
        if use_net:
            return L.make_config(nq, self.ng(nq), box, a_init, 1.0, n_steps, flags=L.FLAG_LEARNED, net=self.net)
        return L.make_config(nq, self.ng(nq), box, a_init, 1.0, n_steps, flags=L.FLAG_LEARNED,
                             net=L.make_net(None, None, self.filter))

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


class FilterFit:
    """Normal equations of the least-squares radial filter, one system per
    filter row (the gathered 1x-mesh force is linear in the node values)."""

    def __init__(self, corr: LearnedCorrection, nq: int, box: float):
        self.corr, self.nq, self.box = corr, nq, box
        na, nb = corr.filter.shape
        self.cfg = L.make_config(nq, corr.ng(nq), box, 0.05)
        self.sim = Simulation(self.cfg, device=corr.device)
        self.sim.init_tables()
        self.basis = torch.empty((nb, 3 * nq**3), dtype=torch.float32, device=corr.device)
        self.ATA = torch.zeros((na, nb, nb), dtype=torch.float64, device=corr.device)
        self.ATy = torch.zeros((na, nb), dtype=torch.float64, device=corr.device)
        self.count = [0] * na

    def add(self, d, a: float, target):
        """Accumulate one configuration: positions d, scale factor a, fine force."""
        na, nb = self.corr.filter.shape
        r = filter_row(a, na)
        self.sim.d.copy_(d)
        L.cola_filter_accumulate(self.cfg, self.sim.state, a, target, nb, self.basis, self.ATA[r], self.ATy[r],
                                 self.sim.ws)
        self.count[r] += 1

    def solve(self, ridge: float = 1e-6):
        na, nb = self.corr.filter.shape
        for r in range(na):
            if self.count[r]:
                L.cola_filter_solve(self.ATA[r], self.ATy[r], nb, ridge, self.corr.filter[r])
        torch.cuda.synchronize()
        return self.corr.filter.clone()


def fit_filter(corr: LearnedCorrection, samples, nq: int, box: float, ridge: float = 1e-6):
    """Least-squares radial filter over stored samples (normal equations summed per row)."""
    fit = FilterFit(corr, nq, box)
    for s in samples:
        fit.add(s.d, s.a, s.force)
    return fit.solve(ridge)


def output_node(a_out: float, a_nodes) -> int:
    """Node whose positions a snapshot at a_out drifts from: the last node
    a_j <= a_out (the final node for a_out >= a_final)."""
    return int(np.searchsorted(np.asarray(a_nodes), a_out + 1e-12, side="right") - 1)


def fit_filter_runs(corr: LearnedCorrection, seeds, nq: int, box: float, m_fine: int = 3, a_init=0.05, n_steps=40,
                    ridge: float = 1e-6, keep_nodes=(), device="cuda", outputs=(1.0,)):
    """Least-squares filter from plain runs at PM_grid = m_fine, accumulated at
    every node of every run without storing the configurations.  Returns the
    Samples at keep_nodes (for the net) and each run's P(k) on an nq^3 mesh at
    the scale factors `outputs` (snapshot drift between nodes), {seed: [(a, k,
    P), ...]}, as by-products."""
    fit = FilterFit(corr, nq, box)
    cfg = L.make_config(nq, m_fine * nq, box, a_init, 1.0, n_steps)
    sim = Simulation(cfg, device=device)
    kept, final = [], {}
    for seed in seeds:
        sim.ic(seed)
        tab = sim.table()[:, 0].cpu().numpy()
        at = {output_node(a, tab): a for a in outputs}
        final[seed] = []
        for j in range(n_steps):
            a = float(tab[j])
            if j in at and j < n_steps - 1:
                k, p, _ = sim.power(nq, a_out=at[j], node=j)
                final[seed].append((at[j], k.cpu().numpy(), p.cpu().numpy()))
            target = sim.force(a)
            fit.add(sim.d, a, target)
            if j in keep_nodes:
                kept.append(Sample(sim.d.clone(), a, target.clone()))
            sim.step(j)
        if n_steps - 1 in at:
            k, p, _ = sim.power(nq, a_out=at[n_steps - 1], node=n_steps - 1)
            final[seed].append((at[n_steps - 1], k.cpu().numpy(), p.cpu().numpy()))
    fit.solve(ridge)
    del sim
    return kept, final


def pk_deviation(k, p, p_ref, kmax: float = 1.0):
    """Mean |P / P_ref - 1| over the bins with k <= kmax."""
    sel = k <= kmax
    return float(np.mean(np.abs(p[sel] / p_ref[sel] - 1.0)))


def golden_section(f, lo: float, hi: float, iters: int = 8):
    """Minimum of a unimodal f on [lo, hi] by golden-section search: iters + 2
    evaluations, the bracket shrinking by 0.618 per iteration.  Returns (x, f(x))."""
    r = (np.sqrt(5.0) - 1.0) / 2.0
    x1, x2 = hi - r * (hi - lo), lo + r * (hi - lo)
    f1, f2 = f(x1), f(x2)
    for _ in range(iters):
        if f1 < f2:
            hi, x2, f2 = x2, x1, f1
            x1 = hi - r * (hi - lo)
            f1 = f(x1)
        else:
            lo, x1, f1 = x1, x2, f2
            x2 = lo + r * (hi - lo)
            f2 = f(x2)
    return (x1, f1) if f1 < f2 else (x2, f2)


def boost_shape(na: int, nb: int, a_init: float = 0.05, a_final: float = 1.0, device="cpu") -> torch.Tensor:
    """(na, nb) shape of the calibration boost: (a_r / a_final) min(k_b / k_Ny, 1)^2
    for filter row r at a_r (rows spaced linearly from a_init to a_final) and
    node b at k_b = b sqrt(3) k_Ny / (nb - 1); one row (na = 1) gets a_r / a_f = 1."""
    kn = torch.arange(nb, dtype=torch.float64, device=device) * (np.sqrt(3.0) / (nb - 1))
    ar = a_init + torch.arange(na, dtype=torch.float64, device=device) * ((a_final - a_init) / max(na - 1, 1))
    rows = (ar / a_final) if na > 1 else torch.ones_like(ar)
    return rows[:, None] * (torch.clamp(kn, max=1.0) ** 2)[None, :]


def calibrated_filter(base: torch.Tensor, g: float, c: float, shape: torch.Tensor) -> torch.Tensor:
    """T' = (1 + g (T - 1)) (1 + c shape): g scales the fitted filter's departure
    from 1, c adds a boost that grows with k up to k_Ny and with a."""
    return ((1.0 + g * (base.double() - 1.0)) * (1.0 + c * shape)).float()


def calibrate_filter(corr: LearnedCorrection, final, nq: int, box: float, kmax: float = 1.0, rounds: int = 2,
                     device="cuda", use_net: bool = True):
    """Fit the least-squares filter's outcome on the training seeds: with
    T'_r = (1 + g (T_r - 1)) (1 + c (a_r / a_f) (k / k_Ny)^2) for k <= k_Ny (the
    boost held at its k_Ny value beyond; a_r the scale factor of filter row r),
    choose g, c by alternating golden-section searches
    that minimise the mean P(k) deviation, over the seeds and their output
    times, of the corrected coarse runs from the seeds' own fine runs (`final`
    from fit_filter_runs, outputs in increasing a).  Returns (g, c)."""
    na, nb = corr.filter.shape
    base = corr.filter.clone()
    # the sub-cell clustering the boost stands in for grows with time: scale it by a_r / a_final
    shape = boost_shape(na, nb, device=corr.device)
    cfg = corr.config(nq, box, use_net=use_net)
    sim = Simulation(cfg, device=device)

    def apply(g, c):
        corr.filter.copy_(calibrated_filter(base, g, c, shape))

    def objective(g, c):
        apply(g, c)
        dev = []
        tab = None
        for seed, outs in final.items():
            sim.ic(seed)
            if tab is None:
                tab = sim.table()[:, 0].cpu().numpy()
            j = 0
            for a_out, k, p3 in outs:
                node = output_node(a_out, tab)
                sim.run(range(j, node))
                j = node
                _, p, _ = sim.power(nq, a_out=a_out, node=node)
                dev.append(pk_deviation(k, p.cpu().numpy(), p3, kmax))
        return float(np.mean(dev))

    g, c = 1.0, 0.0
    for _ in range(rounds):
        c, _ = golden_section(lambda x: objective(g, x), -0.3, 4.0)
        g, _ = golden_section(lambda x: objective(x, c), 0.0, 3.0)
    apply(g, c)
    torch.cuda.synchronize()
    del sim
    return g, c


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
    """Mean relative L2 force error against the fine force for the plain
    coarse mesh, the coarse mesh with the filter, and the full correction
    (keys name the PM_grid = 1 case)."""
    sims = {
        "plain_1x": Simulation(L.make_config(nq, corr.ng(nq), box, 0.05), device=corr.device),
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
