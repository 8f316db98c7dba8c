"""Python handle over the C ABI: one simulation context on one GPU.

PyTorch provides the device memory (one workspace tensor from its caching
allocator) and the CUDA stream; librmhd.so does all the work. Arrays are
structure-of-arrays float64 [n_var][ny][nx].
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L


def _torch():
    import torch
    return torch


def fp64_fma_rate(device=None):
    """(lane FP64 FMAs per second, SM count) of the device, measured by the
    library's probe (rmhd_fp64_fma_rate) on a stream of its own."""
    torch = _torch()
    lib = L.load()
    dev = torch.device("cuda" if device is None else device)
    with torch.cuda.device(dev):
        st = torch.cuda.Stream(dev)
        rate, sms = C.c_double(), C.c_int()
        code = lib.rmhd_fp64_fma_rate(C.c_void_p(st.cuda_stream), C.byref(rate), C.byref(sms))
    if code != L.RMHD_OK:
        raise L.RmhdError(code, "rmhd_fp64_fma_rate")
    return rate.value, sms.value


class Sim:
    """One resistive (N_c = 14) or two-fluid (N_c = 18) SRMHD run."""

    def __init__(self, model: int, nx: int, ny: int, xlim, ylim, gamma: float, sigma: float,
                 bc_x: int, bc_y: int, cfl: float = 0.4, mu_e: float = -1.0, mu_p: float = 1.0,
                 kappa: float = 1.0, precision: int = L.FP64, device=None, scheme: int = L.SSP2,
                 nz: int = 1, zlim=(0.0, 1.0), bc_z: int = L.PERIODIC):
        """nz > 1 makes a 3-D grid (resistive model; arrays [var][nz][ny][nx])."""
        torch = _torch()
        self.lib = L.load()
        self.device = torch.device("cuda" if device is None else device)
        self.nz = max(1, nz)
        self.cfg = L.Config(model, nx, ny, xlim[0], xlim[1], ylim[0], ylim[1], gamma, sigma, mu_e, mu_p,
                            kappa, cfl, bc_x, bc_y, precision, scheme, self.nz, bc_z, zlim[1] - zlim[0])
        self.model, self.nx, self.ny = model, nx, ny
        nbytes = C.c_size_t()
        self._check(self.lib.rmhd_workspace_bytes(C.byref(self.cfg), C.byref(nbytes)), None)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            # a stream of its own: the library captures its step in a CUDA graph,
            # which the legacy default stream does not allow
            self.stream = torch.cuda.Stream(self.device)
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self.h = C.c_void_p()
        self._check(self.lib.rmhd_create(C.byref(self.h), C.byref(self.cfg), C.c_void_p(self.stream.cuda_stream),
                                         C.c_void_p(self.workspace.data_ptr()), nbytes.value), None)

    @property
    def shape(self):
        nz = getattr(self, "nz", 1)
        return (nz, self.ny, self.nx) if nz > 1 else (self.ny, self.nx)

    @classmethod
    def batch(cls, workloads, precision: int = L.FP64, device=None):
        """One context for many independent 1-D runs (same model, x-range,
        Gamma, boundaries; own size and sigma), packed along x."""
        return BatchSim(workloads, precision, device)

    @classmethod
    def from_workload(cls, wl, precision: int = L.FP64, device=None, scheme: int = L.SSP2):
        s = cls(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y, wl.cfl,
                wl.mu_e, wl.mu_p, wl.kappa, precision, device, scheme, wl.nz, wl.zlim, wl.bc_z)
        s.set_prims(wl.prims)
        return s

    # -------------------------------------------------------------- plumbing
    def _check(self, code, what):
        if code != L.RMHD_OK:
            msg = self.lib.rmhd_last_error(self.h).decode() if what is not None and self.h else ""
            raise L.RmhdError(code, msg or str(what))

    @property
    def nc(self):
        return 14 if self.model == L.RESISTIVE else 18

    @property
    def np(self):
        return 11 if self.model == L.RESISTIVE else 16

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.rmhd_destroy(h)
            self.h = None

    def _ptr(self, a, nvar, writable):
        """(pointer, where, keepalive) for a numpy array or a CUDA tensor."""
        torch = _torch()
        n = nvar * self.nx * self.ny * getattr(self, "nz", 1)
        if isinstance(a, torch.Tensor):
            assert a.is_cuda and a.dtype == torch.float64 and a.is_contiguous() and a.numel() == n
            # order the library's stream after the producer of `a` on torch's stream
            self.stream.wait_stream(torch.cuda.current_stream(a.device))
            return C.c_void_p(a.data_ptr()), L.DEVICE, a
        assert isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous and a.size == n
        if writable:
            assert a.flags.writeable
        return C.c_void_p(a.ctypes.data), L.HOST, a

    # -------------------------------------------------------------- API
    def set_prims(self, prims):
        if isinstance(prims, np.ndarray):
            prims = np.ascontiguousarray(prims, dtype=np.float64)
        p, where, _keep = self._ptr(prims, self.np, False)
        self._check(self.lib.rmhd_set_prims(self.h, p, where), "set_prims")

    def set_cons(self, cons):
        if isinstance(cons, np.ndarray):
            cons = np.ascontiguousarray(cons, dtype=np.float64)
        p, where, _keep = self._ptr(cons, self.nc, False)
        self._check(self.lib.rmhd_set_cons(self.h, p, where), "set_cons")

    @property
    def nw(self):
        return 5 if self.model == L.RESISTIVE else 10

    def get_state(self, out=None):
        """Checkpoint for a bitwise restart: N_c + N_w planes (the conserved
        state, then the primitives the next stage solve starts from)."""
        if out is None:
            out = np.empty((self.nc + self.nw,) + self.shape)
        p, where, _keep = self._ptr(out, self.nc + self.nw, True)
        self._check(self.lib.rmhd_get_state(self.h, p, where), "get_state")
        return out

    def set_state(self, state):
        if isinstance(state, np.ndarray):
            state = np.ascontiguousarray(state, dtype=np.float64)
        p, where, _keep = self._ptr(state, self.nc + self.nw, False)
        self._check(self.lib.rmhd_set_state(self.h, p, where), "set_state")

    def prims(self, out=None):
        if out is None:
            out = np.empty((self.np,) + self.shape)
        p, where, _keep = self._ptr(out, self.np, True)
        self._check(self.lib.rmhd_get_prims(self.h, p, where), "get_prims")
        return out

    def cons(self, out=None):
        if out is None:
            out = np.empty((self.nc,) + self.shape)
        p, where, _keep = self._ptr(out, self.nc, True)
        self._check(self.lib.rmhd_get_cons(self.h, p, where), "get_cons")
        return out

    def step(self, dt: float = 0.0, nsteps: int = 1) -> float:
        t = C.c_double()
        self._check(self.lib.rmhd_imex_step(self.h, float(dt), int(nsteps), C.byref(t)), "imex_step")
        return t.value

    def check(self):
        self._check(self.lib.rmhd_check(self.h), "check")

    def record(self, nsteps: int, ckpt_every: int = 10):
        """Arm recording of the next `nsteps` steps for the discrete adjoint
        (call right after set_prims). The checkpoint workspace is a torch tensor."""
        torch = _torch()
        nbytes = C.c_size_t()
        self._check(self.lib.rmhd_recording_bytes(self.h, nsteps, ckpt_every, C.byref(nbytes)), "recording_bytes")
        self.rec_workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
        self._check(self.lib.rmhd_record(self.h, nsteps, ckpt_every, C.c_void_p(self.rec_workspace.data_ptr()),
                                         nbytes.value), "record")

    def adjoint(self, dJ_dcons, out=None):
        """Reverse the recorded steps: dJ/dq(final) -> (dJ/d prims0, dJ/d sigma)."""
        if isinstance(dJ_dcons, np.ndarray):
            dJ_dcons = np.ascontiguousarray(dJ_dcons, dtype=np.float64)
        if out is None:
            out = np.empty((self.np,) + self.shape)
        pin, wi, _k1 = self._ptr(dJ_dcons, self.nc, False)
        pout, wo, _k2 = self._ptr(out, self.np, True)
        gs = C.c_double()
        self._check(self.lib.rmhd_adjoint_step(self.h, pin, wi, pout, wo, C.byref(gs)), "adjoint_step")
        return out, gs.value

    def set_profiling(self, on: bool):
        self._check(self.lib.rmhd_set_profiling(self.h, int(bool(on))), "set_profiling")

    def kernel_times(self) -> dict:
        """{kind: (total ms, launches)} since profiling was enabled (synchronises)."""
        ms, n = (C.c_double * 3)(), (C.c_int * 3)()
        self._check(self.lib.rmhd_kernel_times(self.h, ms, n), "kernel_times")
        return {k: (ms[i], n[i]) for i, k in enumerate(("stage", "flux1", "flux2"))}

    def set_solver_stats(self, on: bool):
        """Start (clearing the counts) or stop counting stage solves into histograms."""
        self._check(self.lib.rmhd_set_solver_stats(self.h, int(bool(on))), "set_solver_stats")

    def solver_stats(self) -> dict:
        """Histograms since the last read: {"fp32_iterations": {k: solves}, "fp64_passes": {k: solves},
        "starts": {"explicit": n, "ideal_limit": n, "continuation": n, "failed": n}}."""
        h = (C.c_ulonglong * 44)()
        self._check(self.lib.rmhd_solver_stats(self.h, h), "solver_stats")
        return {"fp32_iterations": {k: int(h[k]) for k in range(1, 32) if h[k]},
                "fp64_passes": {k: int(h[32 + k - 1]) for k in range(1, 9) if h[32 + k - 1]},
                "starts": {k: int(h[40 + i]) for i, k in enumerate(("explicit", "ideal_limit", "continuation",
                                                                    "failed"))}}

    def set_first_start(self, start: int):
        """Begin every stage solve at start 0 (default), 1 (ideal-MHD limit) or 2 (continuation)."""
        self._check(self.lib.rmhd_set_first_start(self.h, int(start)), "set_first_start")

    def set_refinement_cap(self, passes: int):
        """Cap the FP64 refinement passes of the stage solves (0: default); 1 forces RMHD_ERR_NEWTON."""
        self._check(self.lib.rmhd_set_refinement_cap(self.h, int(passes)), "set_refinement_cap")

    def diagnostics(self) -> dict:
        out = (C.c_double * 8)()
        self._check(self.lib.rmhd_diagnostics(self.h, out), "diagnostics")
        keys = ("sum_D", "sum_tau", "sum_Sx", "sum_Bx", "sum_charge", "max_v", "nonfinite", "dt_cfl")
        return dict(zip(keys, list(out)))


class BatchSim(Sim):
    """Batched ensemble of 1-D runs in one context (rmhd_create_batch)."""

    def __init__(self, workloads, precision: int = L.FP64, device=None):
        torch = _torch()
        self.lib = L.load()
        w0 = workloads[0]
        for w in workloads:
            assert w.ny == 1 and w.model == w0.model and w.gamma == w0.gamma and w.xlim == w0.xlim
            assert (w.bc_x, w.cfl, w.kappa, w.mu_e, w.mu_p) == (w0.bc_x, w0.cfl, w0.kappa, w0.mu_e, w0.mu_p)
        self.device = torch.device("cuda" if device is None else device)
        self.runs = list(workloads)
        self.run_nx = np.array([w.nx for w in workloads], dtype=np.int32)
        self.offsets = np.concatenate([[0], np.cumsum(self.run_nx)])
        self.model, self.nx, self.ny = w0.model, int(self.run_nx.sum()), 1
        self.cfg = L.Config(w0.model, 1, 1, w0.xlim[0], w0.xlim[1], 0.0, 1.0, w0.gamma, w0.sigma, w0.mu_e, w0.mu_p,
                            w0.kappa, w0.cfl, w0.bc_x, w0.bc_y, precision)
        nx_c = (C.c_int * len(workloads))(*self.run_nx.tolist())
        sig_c = (C.c_double * len(workloads))(*[w.sigma for w in workloads])
        nbytes = C.c_size_t()
        self.h = C.c_void_p()
        self._check(self.lib.rmhd_batch_workspace_bytes(C.byref(self.cfg), len(workloads), nx_c, C.byref(nbytes)), None)
        with torch.cuda.device(self.device):
            self.workspace = torch.empty(nbytes.value, dtype=torch.uint8, device=self.device)
            self.stream = torch.cuda.Stream(self.device)
            self.stream.wait_stream(torch.cuda.current_stream(self.device))
        self._check(self.lib.rmhd_create_batch(C.byref(self.h), C.byref(self.cfg), len(workloads), nx_c, sig_c,
                                               C.c_void_p(self.stream.cuda_stream),
                                               C.c_void_p(self.workspace.data_ptr()), nbytes.value), None)
        self.set_prims(self.pack([w.prims for w in workloads]))

    def pack(self, arrays):
        """Concatenate per-run [n_var][1][nx_r] arrays along x."""
        return np.ascontiguousarray(np.concatenate([a.reshape(a.shape[0], 1, -1) for a in arrays], axis=2))

    def unpack(self, packed):
        """Split a packed [n_var][1][sum nx] array into per-run arrays."""
        return [packed[:, :, self.offsets[r]:self.offsets[r + 1]] for r in range(len(self.runs))]

    def autotune(self):
        ch = (C.c_int * 3)()
        self._check(self.lib.rmhd_autotune(self.h, ch), "autotune")
        return {"tile_x": ch[0], "flux_ctas": ch[1], "stage_threads": ch[2]}
