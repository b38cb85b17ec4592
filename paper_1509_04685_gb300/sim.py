"""Torch-allocated buffers around the C ABI: a Simulation owns the particle
state (four SoA float32 tensors of shape (3, nq^3)) and the workspace, and
forwards every call to the library.  No arithmetic of the method happens here."""
from __future__ import annotations

import numpy as np
import torch

from . import _lib as L


class Simulation:
    def __init__(self, cfg: L.cola_config, device="cuda", stream=None):
        self.cfg = cfg
        self.device = torch.device(device)
        self.np = cfg.nq ** 3
        self.ws_bytes = L.cola_workspace_size(cfg)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        f = lambda: torch.zeros((3, self.np), dtype=torch.float32, device=self.device)
        self.d, self.v, self.psi1, self.psi2 = f(), f(), f(), f()
        self.state = L.make_state(self.d, self.v, self.psi1, self.psi2)
        self.stream = stream
        self.node = 0

    def init_tables(self):
        L.cola_init(self.cfg, self.ws, self.stream)

    def ic(self, seed: int):
        L.cola_ic_2lpt(self.cfg, seed, self.state, self.ws, self.stream)
        self.node = 0

    def load_state(self, d, v, psi1, psi2):
        for dst, src in ((self.d, d), (self.v, v), (self.psi1, psi1), (self.psi2, psi2)):
            dst.copy_(torch.as_tensor(src).reshape(3, -1))

    def save_checkpoint(self, path: str):
        """Write the run (config identity, next node, d, v, psi1, psi2) to a file
        through cola_checkpoint_save."""
        buf = torch.empty(L.cola_checkpoint_bytes(self.cfg), dtype=torch.uint8, pin_memory=True)
        L.cola_checkpoint_save(self.cfg, self.state, self.node, buf, self.stream)
        with open(path, "wb") as f:
            f.write(buf.numpy().tobytes())

    def load_checkpoint(self, path: str):
        """Resume a run saved by save_checkpoint: rebuild the workspace tables
        (cola_init), load the state and the next node."""
        n = L.cola_checkpoint_bytes(self.cfg)
        buf = torch.empty(n, dtype=torch.uint8, pin_memory=True)
        with open(path, "rb") as f:
            data = f.read()
        if len(data) != n:
            raise L.ColaError(-1, "load_checkpoint: file size")
        buf.numpy()[:] = np.frombuffer(data, dtype=np.uint8)
        self.init_tables()
        self.node = L.cola_checkpoint_load(self.cfg, buf, self.state, self.stream)

    def step(self, j: int):
        L.cola_step(self.cfg, self.state, j, self.ws, self.stream)
        self.node = min(j + 1, self.cfg.n_steps - 1)

    def step_host(self, host: L.cola_state, j: int):
        """Node j of a state held in host memory (cola_step_host): host's four
        arrays are copied in, d and v are copied back into them."""
        L.cola_step_host(self.cfg, host, self.state, j, self.ws, self.stream)
        self.node = min(j + 1, self.cfg.n_steps - 1)

    def fof(self, b: float = 0.2, min_members: int = 101):
        """Friends-of-friends groups of the current positions: (group label of
        every particle, halo roots, halo sizes) as device tensors, halos of at
        least min_members particles ordered by root."""
        if getattr(self, "fws", None) is None:
            self.fws = torch.empty(L.cola_fof_workspace_size(self.cfg), dtype=torch.uint8, device=self.device)
        group = torch.empty(self.np, dtype=torch.int32, device=self.device)
        L.cola_fof(self.cfg, self.state, b, group, self.fws, self.stream)
        cap = self.np // max(1, min_members) + 1
        roots = torch.empty(cap, dtype=torch.int32, device=self.device)
        sizes = torch.empty(cap, dtype=torch.int32, device=self.device)
        n = torch.zeros(1, dtype=torch.int64, device=self.device)
        L.cola_fof_halos(self.cfg, group, min_members, roots, sizes, n, self.fws, self.stream)
        nh = int(n.item())
        return group, roots[:nh], sizes[:nh]

    def mass_function(self, sizes, lo: float, dlog: float, nbins: int):
        """Halo counts per bin of log10 M (Warren masses) for halo sizes `sizes`."""
        n = torch.tensor([sizes.numel()], dtype=torch.int64, device=self.device)
        counts = torch.empty(nbins, dtype=torch.int64, device=self.device)
        L.cola_mass_function(self.cfg, sizes, n, sizes.numel(), lo, dlog, nbins, counts, self.stream)
        return counts

    def run(self, steps=None):
        for j in range(self.cfg.n_steps) if steps is None else steps:
            self.step(j)

    def force(self, a: float, out=None):
        out = torch.empty((3, self.np), dtype=torch.float32, device=self.device) if out is None else out
        L.cola_pm_force(self.cfg, self.state, a, out, self.ws, self.stream)
        return out

    def density(self):
        ng = self.cfg.ng
        out = torch.empty((ng, ng, ng), dtype=torch.float32, device=self.device)
        L.cola_density(self.cfg, self.state, out, self.ws, self.stream)
        return out

    def power(self, ng_pk: int, a_out: float | None = None, flags: int = 0, node: int | None = None):
        nb = ng_pk // 2
        k, p, n = (torch.zeros(nb, dtype=torch.float64, device=self.device) for _ in range(3))
        node = self.node if node is None else node
        a = self.table()[node, 0].item() if a_out is None else a_out
        L.cola_power_spectrum(self.cfg, self.state, node, a, ng_pk, flags, k, p, n, self.ws, self.stream)
        return k, p, n

    def multipoles(self, ng_pk: int, a_out: float | None = None, flags: int = 0, node: int | None = None):
        """Redshift-space P0, P2, P4 about the z axis: (k, p0, p2, p4, nmodes)."""
        nb = ng_pk // 2
        k, p0, p2, p4, n = (torch.zeros(nb, dtype=torch.float64, device=self.device) for _ in range(5))
        node = self.node if node is None else node
        a = self.table()[node, 0].item() if a_out is None else a_out
        L.cola_power_multipoles(self.cfg, self.state, node, a, ng_pk, flags, k, p0, p2, p4, n, self.ws, self.stream)
        return k, p0, p2, p4, n

    def table(self):
        out = torch.empty((self.cfg.n_steps, 12), dtype=torch.float64, device=self.device)
        L.cola_step_table(self.cfg, out, self.ws, self.stream)
        return out

    def status(self) -> int:
        return L.cola_status(self.ws, self.stream)
