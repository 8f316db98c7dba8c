"""Domain decomposition along y: slabs of one 2-D grid, stepped phase by phase
with a halo exchange before every flux pass (multi-GPU runs are future work
in the paper, Sec. 3.1 and Sec. 5; this is the exchange step they need).

Each slab is a context of the C ABI (rmhd_create_slab) holding rows
[j0, j0 + ny_local) of the global grid. One IMEX step is 4 phases (SSP2(222))
or 6 (SSP3(332)) of rmhd_step_phase. For every stage k:
  1. every slab runs its implicit stage solve (even phase; per cell, no
     neighbour data);
  2. every slab packs the first two and the last two rows of its stage state
     (rmhd_halo_pack);
  3. slab s receives the last rows of slab s - 1 into its lower halo and the
     first rows of slab s + 1 into its upper halo (cyclically on a periodic
     grid; a global outflow boundary has no halo) and unpacks them;
  4. every slab runs its flux pass (odd phase).
With the halos exchanged every slab's rows equal the undecomposed run's, bit
for bit.

`LocalSlabs` keeps all slabs of a grid on one GPU and one CUDA stream (the
exchange is a device copy). `DistSlab` is one slab per process of a
torch.distributed group: the exchange is point-to-point send/receive (NCCL on
GPUs, gloo on the host), ordered on the slab's stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .sim import Sim, _torch


def neighbours(rank: int, world: int, periodic: bool):
    """(lower, upper) neighbour ranks of slab `rank` of `world` slabs ordered
    along y; None where the slab touches a global outflow boundary."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic else None)
    hi = rank + 1 if rank < world - 1 else (0 if periodic else None)
    return lo, hi


def split_rows(ny: int, parts: int):
    """Row counts of `parts` slabs covering ny rows as evenly as possible."""
    base, extra = divmod(ny, parts)
    return [base + (1 if s < extra else 0) for s in range(parts)]


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic: bool, group=None):
    """Point-to-point halo exchange with the two neighbours (torch.distributed).

    Upward first (every slab sends its last rows up and receives its lower
    halo from below), then downward (first rows down, upper halo from above).
    Posting the two directions in this order on every rank matches each send
    with its receive also when one peer is both neighbours (two periodic
    slabs), and in backends that match by posting order only. A slab that is
    its own neighbour (one periodic slab) copies locally. Returns the pending
    requests (wait on them before the flux pass)."""
    import torch.distributed as dist
    lo, hi = neighbours(rank, world, periodic)
    if world == 1:
        if lo is not None:
            recv_lo.copy_(send_hi)
        if hi is not None:
            recv_hi.copy_(send_lo)
        return []
    ops = []
    if hi is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, hi, group, tag=0))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lo, group, tag=0))
    if lo is not None:
        ops.append(dist.P2POp(dist.isend, send_lo, lo, group, tag=1))
    if hi is not None:
        ops.append(dist.P2POp(dist.irecv, recv_hi, hi, group, tag=1))
    return dist.batch_isend_irecv(ops) if ops else []


class SlabSim(Sim):
    """One slab [j0, j0 + ny_local) of the 2-D grid of workload-like global
    parameters (a context of rmhd_create_slab)."""

    def __init__(self, model, nx, ny_global, j0, ny_local, xlim, ylim, gamma, sigma, bc_x, bc_y, cfl=0.4,
                 mu_e=-1.0, mu_p=1.0, kappa=1.0, precision=L.FP64, device=None, scheme=L.SSP2, stream=None):
        torch = _torch()
        self.lib = L.load()
        self.device = torch.device("cuda" if device is None else device)
        self.nz = 1
        self.cfg = L.Config(model, nx, ny_global, xlim[0], xlim[1], ylim[0], ylim[1], gamma, sigma, mu_e, mu_p,
                            kappa, cfl, bc_x, bc_y, precision, scheme, 1, L.PERIODIC, 1.0)
        self.model, self.nx, self.ny = model, nx, ny_local
        self.j0, self.ny_global = j0, ny_global
        self.h = C.c_void_p()
        nbytes = C.c_size_t()
        self._check(self.lib.rmhd_slab_workspace_bytes(C.byref(self.cfg), j0, ny_local, C.byref(nbytes)), None)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            self.stream = stream if stream is not None else torch.cuda.Stream(self.device)
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.rmhd_create_slab(C.byref(self.h), C.byref(self.cfg), j0, ny_local,
                                              C.c_void_p(self.stream.cuda_stream),
                                              C.c_void_p(self.workspace.data_ptr()), nbytes.value), None)
        n = C.c_size_t()
        self._check(self.lib.rmhd_halo_doubles(self.h, C.byref(n)), "halo_doubles")
        self.halo_doubles = n.value
        self.phases = 6 if scheme == L.SSP3 else 4

    @classmethod
    def of_workload(cls, wl, j0, ny_local, precision=L.FP64, device=None, scheme=L.SSP2, stream=None):
        assert wl.nz == 1 and wl.ny > 1
        return cls(wl.model, wl.nx, wl.ny, j0, ny_local, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y,
                   wl.cfl, wl.mu_e, wl.mu_p, wl.kappa, precision, device, scheme, stream)

    def step_phase(self, dt: float, phase: int) -> float:
        t = C.c_double()
        self._check(self.lib.rmhd_step_phase(self.h, float(dt), int(phase), C.byref(t)), "step_phase")
        return t.value

    def halo_pack(self, lo, hi):
        self._check(self.lib.rmhd_halo_pack(self.h, C.c_void_p(lo.data_ptr() if lo is not None else 0),
                                            C.c_void_p(hi.data_ptr() if hi is not None else 0)), "halo_pack")

    def halo_unpack(self, lo, hi):
        self._check(self.lib.rmhd_halo_unpack(self.h, C.c_void_p(lo.data_ptr() if lo is not None else 0),
                                              C.c_void_p(hi.data_ptr() if hi is not None else 0)), "halo_unpack")

    def halo_buffers(self):
        """Four device buffers (send lo, send hi, recv lo, recv hi) of one halo side each."""
        torch = _torch()
        return [torch.empty(self.halo_doubles, dtype=torch.float64, device=self.device) for _ in range(4)]


class LocalSlabs:
    """All slabs of one 2-D grid on one GPU, sharing one CUDA stream."""

    def __init__(self, wl, rows, precision=L.FP64, device=None, scheme=L.SSP2):
        torch = _torch()
        assert sum(rows) == wl.ny
        self.wl = wl
        self.periodic = wl.bc_y == L.PERIODIC
        dev = torch.device("cuda" if device is None else device)
        self.stream = torch.cuda.Stream(dev)
        self.slabs, j0 = [], 0
        for ny in rows:
            self.slabs.append(SlabSim.of_workload(wl, j0, ny, precision, dev, scheme, self.stream))
            j0 += ny
        self.bufs = [s.halo_buffers() for s in self.slabs]

    def set_state(self, state):
        """The full-state checkpoint of the whole grid ([N_c + N_w][ny][nx]), split by rows."""
        for s in self.slabs:
            s.set_state(np.ascontiguousarray(state[:, s.j0:s.j0 + s.ny]))

    def _exchange(self):
        torch = _torch()
        n = len(self.slabs)
        with torch.cuda.stream(self.stream):
            for s, b in zip(self.slabs, self.bufs):
                s.halo_pack(b[0], b[1])
            for k, (s, b) in enumerate(zip(self.slabs, self.bufs)):
                lo, hi = neighbours(k, n, self.periodic)
                if lo is not None:
                    b[2].copy_(self.bufs[lo][1])
                if hi is not None:
                    b[3].copy_(self.bufs[hi][0])
                s.halo_unpack(b[2] if lo is not None else None, b[3] if hi is not None else None)

    def step(self, dt: float, nsteps: int = 1):
        for _ in range(nsteps):
            for p in range(self.slabs[0].phases):
                if p % 2 == 1:
                    self._exchange()
                for s in self.slabs:
                    s.step_phase(dt, p)

    def check(self):
        for s in self.slabs:
            s.check()

    def _gather(self, fn):
        return np.concatenate([fn(s) for s in self.slabs], axis=1)

    def cons(self):
        return self._gather(lambda s: s.cons())

    def prims(self):
        return self._gather(lambda s: s.prims())

    def get_state(self):
        return self._gather(lambda s: s.get_state())


class DistSlab:
    """This process's slab of a grid decomposed over a torch.distributed group
    (rank r holds the r-th block of rows); halos move by point-to-point
    send/receive on the slab's stream."""

    def __init__(self, wl, rank, world, precision=L.FP64, device=None, scheme=L.SSP2, group=None):
        rows = split_rows(wl.ny, world)
        j0 = sum(rows[:rank])
        self.rank, self.world, self.group = rank, world, group
        self.periodic = wl.bc_y == L.PERIODIC
        self.slab = SlabSim.of_workload(wl, j0, rows[rank], precision, device, scheme)
        self.bufs = self.slab.halo_buffers()

    def step(self, dt: float, nsteps: int = 1):
        torch = _torch()
        s, b = self.slab, self.bufs
        lo, hi = neighbours(self.rank, self.world, self.periodic)
        for _ in range(nsteps):
            for p in range(s.phases):
                if p % 2 == 1:
                    with torch.cuda.stream(s.stream):
                        s.halo_pack(b[0], b[1])
                        for r in exchange(b[0], b[1], b[2], b[3], self.rank, self.world, self.periodic, self.group):
                            r.wait()
                        s.halo_unpack(b[2] if lo is not None else None, b[3] if hi is not None else None)
                s.step_phase(dt, p)
