#!/usr/bin/env python3
"""Benchmark of the SSP2(222) IMEX step for resistive SRMHD on GB300.

Workload: 2-D resistive SRMHD Kelvin-Helmholtz shear layer, 1024 x 1024 cells,
periodic, Gamma = 4/3, sigma = 1e3, seeded synthetic data (the shape of the
paper's KHI test, Sec. 4.4). One "step" = one full SSP2(222) IMEX step (two
implicit per-cell stage solves, two WENO3/LF flux passes, stage combine and
recovery) over all cells. Metric: cell-updates/s.

Printed JSON line: the FP64 form is `value`; the mixed form (FP32 flux
arithmetic, FP64 source solve) is under "mixed" and the float-float form
(flux arithmetic in pairs of FP32 numbers, FP64 source solve) under
"floatfloat", each with its error against the FP64 result; "e2e" is the same metric through the C ABI with host buffers
(prims uploaded and read back every step); "roofline" is for the dominant
kernel, timed with CUDA events inside the timed region; "cpu_baseline" is the
FP64 CPU oracle on the host cores on a bounded sample of the same workload.

Multi-GPU (torchrun): the headline FP64 step runs on a grid decomposed along y,
one slab per GPU, with the two halo rows of every variable exchanged by NCCL
point-to-point before each flux pass (weak scaling: rank r holds the r-th copy
of the 1024^2 shear layer stacked along y, a periodic grid of 1024 x 1024N
cells). `--replicas` runs independent replicas instead. The other workloads run
as replicas. Times are the max over ranks.

`--impl reference` times the CPU oracle instead (the reference arm of this
repository: there is no reference implementation to install).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s per IMEX step, FP64 vs mixed, % HBM roofline; adjoint/fwd cost"
UNIT = "cell-updates/s"
def workload_name(n: int = 1024) -> str:
    return (f"khi-2d-{n}x{n} (resistive SRMHD Kelvin-Helmholtz, periodic, Gamma=4/3, sigma=1e3, SSP2(222), "
            "WENO3+LF)")

# Algorithmic FP64 operations (+, -, x, /, sqrt; one flop each) per interior
# cell of the flux passes of a 2-D periodic grid, counted by the op-counting
# build of the CPU oracle (oracle/opcount.py: each cell's flux once per
# direction, each face's two WENO3 reconstructions once per component, the
# source and the stage combinations; a test recomputes them): pass 1 has two
# outputs (r2, acc), pass 2 one (q^{n+1}).
ALG_FP64_FLOPS_PER_CELL = {"flux1": 1918, "flux2": 1880, "tf_flux1": 2556, "tf_flux2": 2502}
# FP64 arithmetic instructions the kernels themselves issue (dadd, dmul, dfma;
# one each) per interior cell on a 2-D grid, counted by ncu's
# smsp__sass_thread_inst_executed_op_{dadd,dmul,dfma} on a 512x512 KHI step.
FP64_INST_PER_CELL = {"stage": 184.0, "flux1": 668.5, "flux2": 654.5}
# DRAM bytes (read + write) per cell and launch of the same kernels, from an
# ncu capture of the 512x512 KHI step (dram__bytes_read.sum + write.sum): the
# reads scale with the cells; at that size part of the writes is still in L2
# when a kernel ends, so the full-size writes are somewhat higher.
DRAM_BYTES_PER_CELL = {"stage": 126.6, "flux1": 484.9, "flux2": 365.1}
# Algorithmic HBM bytes per cell for each kernel (read once + written once; the
# stage also writes J, Z and p + (E^2 + B^2)/2 of its result for the flux passes).
BYTES_PER_CELL = {"stage": 8 * (14 + 1 + 14 + 5 + 5), "flux1": 8 * (19 + 5 + 14 + 28),
                  "flux2": 8 * (19 + 5 + 14 + 19)}


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return float(d.get("hbm_gbs", 6800.0)), "measured", float(d.get("sm_max_mhz", 2070.0))
    return 6800.0, "fallback", 2070.0


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if self.proc is None or not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], None, set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.path)
        sm.sort()
        med = sm[len(sm) // 2] if sm else None
        return {"sm_mhz": med, "sm_max_mhz": smax, "reasons": sorted(reasons), "samples": len(sm)}


def natural_scale(model, want, mu_ref=1.0):
    """Per-variable scale used for errors: vector components share one; the
    charge/cleaning fields are scaled by the field magnitude; for two fluids
    the mu-weighted totals (Dbar, Sbar, taubar) by mu_ref times D, S, tau."""
    import numpy as np
    m = np.abs(want).reshape(want.shape[0], -1).max(axis=1)
    s = m.copy()
    bs, es = (5, 8) if model == 0 else (10, 13)
    B, E = want[bs:bs + 3], want[es:es + 3]
    exb = float(np.max(np.sqrt((B * B).sum(axis=0) * (E * E).sum(axis=0))))  # S includes E x B
    if model == 0:
        for a, b in ((1, 4), (5, 8), (8, 11)):
            s[a:b] = m[a:b].max()
        s[1:4] = max(s[1], exb)
        s[11:14] = np.maximum(m[11:14], max(s[5], s[8]))
    else:
        for a, b in ((1, 4), (6, 9), (10, 13), (13, 16)):
            s[a:b] = m[a:b].max()
        s[1:4] = max(s[1], exb)
        s[5] = max(m[5], mu_ref * m[0])
        s[6:9] = max(s[6], mu_ref * s[1])
        s[9] = max(m[9], mu_ref * m[4])
        s[16:18] = np.maximum(m[16:18], max(s[10], s[13]))
    return np.maximum(s, 1e-300)


def rel_l1(model, got, want, mu_ref=1.0):
    """Largest over variables of mean |got - want| / natural scale."""
    import numpy as np
    nv = want.shape[0]
    w3 = want.reshape(nv, -1, 1)
    return float(np.max(np.abs(got - want).reshape(nv, -1).mean(axis=1) / natural_scale(model, w3, mu_ref)))


def reduce_max(x: float, world: int, device: str) -> float:
    """Max of a per-rank value (elapsed time) over all ranks of the process
    group (NCCL on the GPUs; any backend whose device is given)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def cpu_baseline(seconds: float = 15.0):
    """FP64 CPU oracle on the host cores: KHI recipe at 128 x 128 (a bounded
    sample of the benchmark workload), as many steps as fit in ~`seconds`."""
    import oracle as O
    from paper_1808_09721_gb300 import workloads as WL
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    wl = WL.khi(n=128, seed=0)
    s = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    s.set_prims(wl.prims)
    t0 = time.perf_counter()
    s.step(wl.dt, 1)
    t1 = time.perf_counter() - t0
    steps = max(1, min(5000, int(seconds / max(t1, 1e-6))))
    t0 = time.perf_counter()
    s.step(wl.dt, steps)
    el = time.perf_counter() - t0
    value = steps * wl.cells / el
    # one-core figure (the paper's CPU baseline is a single core), short sample
    O.set_threads(1)
    s1 = O.Sim(wl.model, 32, 32, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    s1.set_prims(WL.khi(n=32, seed=0).prims)
    t0 = time.perf_counter()
    s1.step(wl.dt, 2)
    one = 2 * 32 * 32 / (time.perf_counter() - t0)
    O.set_threads(cores)
    return {"value": value, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
            "sample": f"KHI recipe 128x128 periodic, {steps} SSP2(222) steps ({el:.1f} s), all host cores",
            "single_core_value": one}


def run_reference(args, rank, world):
    """--impl reference: the FP64 CPU oracle, each step a bounded sample (one
    SSP2(222) step of the KHI recipe at 96 x 96)."""
    if rank != 0:
        return
    import oracle as O
    from paper_1808_09721_gb300 import workloads as WL
    cores = os.cpu_count() or 1
    O.set_threads(cores)
    wl = WL.khi(n=96, seed=0)
    s = O.Sim(wl.model, wl.nx, wl.ny, wl.xlim, wl.ylim, wl.gamma, wl.sigma, wl.bc_x, wl.bc_y)
    s.set_prims(wl.prims)
    s.step(wl.dt, args.warmup)
    t0 = time.perf_counter()
    s.step(wl.dt, args.steps)
    el = time.perf_counter() - t0
    value = args.steps * wl.cells / el
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": workload_name(args.n), "cells_per_gpu": args.n * args.n,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2: state+workspace > 129 MB"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.get_threads(), "kind": "oracle",
                             "sample": "KHI recipe 96x96 periodic (a window of the workload), one SSP2(222) "
                                       "step per bench step, all host cores"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=("ours", "reference"))
    ap.add_argument("--n", type=int, default=1024, help="grid side (default: the 1024^2 workload)")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU-oracle baseline")
    ap.add_argument("--no-batch", dest="batch", action="store_false", help="skip the batched-ensemble workload")
    ap.add_argument("--no-adjoint", dest="adjoint", action="store_false", help="skip the adjoint-cost workload")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="skip the two-fluid 512^2 and Brio-Wu 1-D workloads")
    ap.add_argument("--replicas", action="store_true",
                    help="N > 1: independent replicas instead of the decomposed grid")
    args = ap.parse_args()
    assert args.warmup >= 3 or args.impl == "reference", "at least 3 warm-up steps"

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch
    import torch.distributed as dist

    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1808_09721_gb300 import build as B
    if rank == 0:
        B.build()
    if world > 1:
        dist.barrier()
    B.build()
    from paper_1808_09721_gb300 import FP64, MIXED, FLOATFLOAT, HOST
    from paper_1808_09721_gb300 import workloads as WL
    from paper_1808_09721_gb300.sim import Sim, fp64_fma_rate

    wl = WL.khi(n=args.n, seed=0)
    K, W = args.steps, args.warmup

    def barrier():
        if world > 1:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        return reduce_max(x, world, f"cuda:{local}")

    def timed_run(precision, profile, w=None, k=None, scheme=0):
        """W warm-up steps, then k timed steps as one CUDA graph per step
        (the production path). With `profile`, k more steps follow with
        per-launch CUDA events (no graph) for the per-kernel times."""
        w = wl if w is None else w
        k = K if k is None else k
        sim = Sim.from_workload(w, precision=precision, device=f"cuda:{local}", scheme=scheme)
        sim.step(w.dt, W)
        sim.check()
        st = sim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(st)
        sim.step(w.dt, k)
        e1.record(st)
        torch.cuda.synchronize()
        barrier()
        ms = e0.elapsed_time(e1)
        sim.check()
        kt = None
        if profile:
            sim.set_profiling(True)
            sim.step(w.dt, k)
            kt = sim.kernel_times()
            sim.set_profiling(False)
            sim.check()
        return sim, max_over_ranks(ms), kt

    with ClockSampler(local) as clk:
        sim64, ms64, kt64 = timed_run(FP64, True)
    clocks = clk.summary()
    simmx, msmx, ktmx = timed_run(MIXED, True)
    q64, qmx = sim64.cons(), simmx.cons()
    rel_l1_mixed = float(np.max(np.abs(qmx - q64).reshape(14, -1).mean(axis=1) / natural_scale(0, q64)))
    del simmx
    # float-float flux form: FP64-class accuracy from the FP32 pipes
    simff, msff, ktff = timed_run(FLOATFLOAT, True)
    qff = simff.cons()
    dff = np.abs(qff - q64).reshape(14, -1)
    rel_linf_ff = float(np.max(dff.max(axis=1) / natural_scale(0, q64)))
    rel_l1_ff = float(np.max(dff.mean(axis=1) / natural_scale(0, q64)))
    del simff

    # N > 1: the headline step on the decomposed grid (slabs along y, NCCL halo exchange)
    decomposed = world > 1 and not args.replicas
    if decomposed:
        from paper_1808_09721_gb300.slabs import DistSlab
        gwl = wl.with_prims(np.concatenate([wl.prims] * world, axis=1), ny=wl.ny * world,
                            ylim=(wl.ylim[0], wl.ylim[0] + world * (wl.ylim[1] - wl.ylim[0])))
        ds = DistSlab(gwl, rank, world, device=f"cuda:{local}")
        init = Sim.from_workload(wl, device=f"cuda:{local}")  # this rank's copy: the same rows, periodic
        ds.slab.set_state(init.get_state())
        del init
        ds.step(wl.dt, W)
        ds.slab.check()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(ds.slab.stream)
        ds.step(wl.dt, K)
        e1.record(ds.slab.stream)
        torch.cuda.synchronize()
        barrier()
        ms64 = max_over_ranks(e0.elapsed_time(e1))
        ds.slab.check()
        del ds

    total_cells = world * wl.cells
    value = total_cells * K / (ms64 * 1e-3)
    value_mx = total_cells * K / (msmx * 1e-3)
    value_ff = total_cells * K / (msff * 1e-3)

    # the other single-grid workloads: two-fluid current sheet 512^2 (FP64 and
    # mixed) and the 1-D Brio-Wu tube (400 cells, launch-bound, 100 steps)
    extra = None
    if args.extra:
        tfw = WL.tf_sheet(n=512, seed=1)
        tf64, ms_tf64, kt_tf64 = timed_run(FP64, True, tfw)
        tfmx, ms_tfmx, kt_tfmx = timed_run(MIXED, True, tfw)
        tfff, ms_tfff, kt_tfff = timed_run(FLOATFLOAT, True, tfw)
        qa, qb, qc = tf64.cons(), tfmx.cons(), tfff.cons()
        l1_tf = float(np.max(np.abs(qb - qa).reshape(qa.shape[0], -1).mean(axis=1) /
                             natural_scale(1, qa, abs(tfw.mu_p))))
        linf_tf_ff = float(np.max(np.abs(qc - qa).reshape(qa.shape[0], -1).max(axis=1) /
                                  natural_scale(1, qa, abs(tfw.mu_p))))
        del tf64, tfmx, tfff
        bw = WL.brio_wu()
        bws, ms_bw, _ = timed_run(FP64, False, bw, 100)
        del bws
        tbw = WL.tf_brio_wu(nx=1600)
        tbws, ms_tbw, _ = timed_run(FP64, False, tbw, 100)
        del tbws
        k3 = WL.khi3d(n=128, seed=0)
        s3d, ms_3d, kt_3d = timed_run(FP64, True, k3)
        s3dm, ms_3dm, _ = timed_run(MIXED, True, k3)
        l1_3d = rel_l1(0, s3dm.cons(), s3d.cons())
        del s3d, s3dm
        s3, ms_s3, kt_s3 = timed_run(FP64, True, None, None, 1)
        s3m, ms_s3m, _ = timed_run(MIXED, True, None, None, 1)
        l1_s3 = rel_l1(0, s3m.cons(), s3.cons())
        del s3, s3m
        extra = {"two_fluid_512": {"fp64": world * tfw.cells * K / (ms_tf64 * 1e-3),
                                   "mixed": world * tfw.cells * K / (ms_tfmx * 1e-3),
                                   "floatfloat": world * tfw.cells * K / (ms_tfff * 1e-3),
                                   "ms_per_step_fp64": ms_tf64 / K, "ms_per_step_mixed": ms_tfmx / K,
                                   "ms_per_step_floatfloat": ms_tfff / K, "rel_linf_floatfloat_vs_fp64": linf_tf_ff,
                                   "kernels_ms_per_launch_floatfloat": {k: v[0] / max(v[1], 1) for k, v in kt_tfff.items()},
                                   "rel_l1_mixed_vs_fp64": l1_tf, "unit": UNIT,
                                   "kernels_ms_per_launch_fp64": {k: v[0] / max(v[1], 1) for k, v in kt_tf64.items()},
                                   "kernels_ms_per_launch_mixed": {k: v[0] / max(v[1], 1) for k, v in kt_tfmx.items()},
                                   "workload": "two-fluid current sheet 512x512, mu=+-1e3, sigma=1e4, periodic"},
                 "khi_1024_ssp3": {"fp64": world * wl.cells * K / (ms_s3 * 1e-3),
                                   "mixed": world * wl.cells * K / (ms_s3m * 1e-3),
                                   "ms_per_step_fp64": ms_s3 / K, "ms_per_step_mixed": ms_s3m / K,
                                   "rel_l1_mixed_vs_fp64": l1_s3,
                                   "unit": UNIT,
                                   "kernels_ms_per_launch_fp64": {k: v[0] / max(v[1], 1) for k, v in kt_s3.items()},
                                   "workload": "KHI 1024x1024 with SSP3(332) (Table 2): 3 implicit stages, 3 flux passes"},
                 "khi3d_128": {"fp64": world * k3.cells * K / (ms_3d * 1e-3),
                               "mixed": world * k3.cells * K / (ms_3dm * 1e-3),
                               "ms_per_step_fp64": ms_3d / K, "ms_per_step_mixed": ms_3dm / K, "unit": UNIT,
                               "rel_l1_mixed_vs_fp64": l1_3d,
                               "kernels_ms_per_launch_fp64": {k: v[0] / max(v[1], 1) for k, v in kt_3d.items()},
                               "workload": "3-D KHI 128^3 periodic, SSP2(222); flux pass = x-y pass + z pass"},
                 "tf_brio_wu_1600": {"fp64": world * tbw.cells * 100 / (ms_tbw * 1e-3), "unit": UNIT,
                                     "us_per_step": 1e3 * ms_tbw / 100,
                                     "workload": "1-D two-fluid Brio-Wu, pair plasma mu=+-1e3, 1600 cells, 100 steps"},
                 "brio_wu_400": {"fp64": world * bw.cells * 100 / (ms_bw * 1e-3), "unit": UNIT,
                                 "us_per_step": 1e3 * ms_bw / 100,
                                 "workload": "1-D Brio-Wu tube, 400 cells, sigma=100, 100 graph-captured steps"}}

    # batched ensemble: 512 independent 1-D shock tubes, N ~ U{100..4096},
    # sigma log-uniform in [1, 1e6], own CFL dt, mixed form, one graph per step
    batch = None
    if args.batch:
        runs = WL.batch_tubes(count=512, seed=2)
        bsim = Sim.batch(runs, precision=MIXED, device=f"cuda:{local}")
        choice = bsim.autotune()
        bsim.step(0.0, W)
        bsim.check()
        bst = bsim.stream
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        torch.cuda.synchronize()
        e0.record(bst)
        bsim.step(0.0, K)
        e1.record(bst)
        torch.cuda.synchronize()
        barrier()
        bms = max_over_ranks(e0.elapsed_time(e1))
        bsim.check()
        bcells = int(bsim.nx)
        # the configuration's whole run: 400 steps of every tube from its initial state
        bsim.set_prims(bsim.pack([w.prims for w in runs]))
        torch.cuda.synchronize()
        e0.record(bst)
        bsim.step(0.0, 400)
        e1.record(bst)
        torch.cuda.synchronize()
        bsim.check()
        full_ms = e0.elapsed_time(e1)
        # error of the mixed form: every tube's 400-step state against the FP64 run
        b64 = Sim.batch(runs, precision=FP64, device=f"cuda:{local}")
        b64.step(0.0, 400)
        b64.check()
        gm, g64 = bsim.unpack(bsim.cons()), b64.unpack(b64.cons())
        l1_batch = max(rel_l1(0, a, b) for a, b in zip(gm, g64))
        del b64
        batch = {"value": world * bcells * K / (bms * 1e-3), "unit": UNIT, "ms_per_step": bms / K,
                 "runs": len(runs), "cells": bcells, "dtype": "f32 flux / f64 source",
                 "full_run_400_steps_s": full_ms * 1e-3, "autotune": choice,
                 "rel_l1_mixed_vs_fp64_max_over_tubes": l1_batch,
                 "workload": "512 1-D resistive shock tubes, N~U{100..4096}, sigma log-uniform [1,1e6], "
                             "Gamma=4/3, own CFL dt, one CUDA graph per step"}
        del bsim

    # discrete adjoint: field loop 256^2, 50 FP64 steps, checkpoints every 10;
    # gradient of sum (B_x^2 + B_y^2 + 2 B_z^2) dV w.r.t. initial prims and sigma
    adjoint = None
    if args.adjoint:
        fl = WL.field_loop(n=256, seed=3, nsteps=50)

        def adjoint_cost(wa, scheme, b0):
            """Forward, recorded forward and adjoint wall times of 50 steps
            (checkpoints every 10); J = sum(Bx^2 + By^2 + 2 Bz^2) dV with B at
            conserved rows b0 .. b0 + 2."""
            fs = Sim.from_workload(wa, device=f"cuda:{local}", scheme=scheme)
            fs.step(wa.dt, 3)
            fs.set_prims(wa.prims)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fs.step(wa.dt, 50)
            fs.check()
            torch.cuda.synchronize()
            t_fwd = time.perf_counter() - t0
            fs.set_prims(wa.prims)
            fs.record(50, 10)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fs.step(wa.dt, 50)
            fs.check()
            torch.cuda.synchronize()
            t_rec = time.perf_counter() - t0
            qN = fs.cons()
            dv = wa.dx * wa.dy
            lam = np.zeros_like(qN)
            lam[b0] = 2.0 * qN[b0] * dv
            lam[b0 + 1] = 2.0 * qN[b0 + 1] * dv
            lam[b0 + 2] = 4.0 * qN[b0 + 2] * dv
            fs.adjoint(lam)  # warm-up (kernel set-up)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            gp, gsig = fs.adjoint(lam)
            torch.cuda.synchronize()
            t_adj = time.perf_counter() - t0
            return {"fwd_s": t_fwd, "recorded_fwd_s": t_rec, "adjoint_s": t_adj,
                    "adjoint_over_fwd": t_adj / t_fwd, "total_over_fwd": (t_rec + t_adj) / t_fwd, "dJ_dsigma": gsig}
        adjoint = adjoint_cost(fl, 0, 5)
        tfa = WL.tf_sheet(n=128, seed=1)
        adjoint.update({"sigma": fl.sigma, "ssp3": adjoint_cost(fl, 1, 5),
                        "workload": "field loop 256x256 periodic, 50 SSP2(222) steps FP64 (and SSP3(332) in "
                                    "'ssp3'), checkpoints every 10, J = sum(Bx^2 + By^2 + 2 Bz^2) dV",
                        "two_fluid": dict(adjoint_cost(tfa, 0, 10), workload="two-fluid current sheet 128x128 "
                                          "periodic (mu = -+1e3, sigma 1e4), 50 SSP2(222) steps FP64, "
                                          "checkpoints every 10, J = sum(Bx^2 + By^2 + 2 Bz^2) dV")})

    # e2e through the C ABI with host buffers: upload prims, one step, read prims back
    pin = torch.empty(wl.prims.size, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.prims.shape)
    pin[...] = wl.prims
    out = torch.empty(wl.prims.size, dtype=torch.float64, pin_memory=True).numpy().reshape(wl.prims.shape)
    e2e_sim = sim64
    for _ in range(2):
        e2e_sim.set_prims(pin)
        e2e_sim.step(wl.dt, 1)
        e2e_sim.prims(out=out)
    barrier()
    t0 = time.perf_counter()
    for _ in range(K):
        e2e_sim.set_prims(pin)
        e2e_sim.step(wl.dt, 1)
        e2e_sim.prims(out=out)
    torch.cuda.synchronize()
    barrier()
    e2e_s = max_over_ranks(time.perf_counter() - t0)
    e2e_value = total_cells * K / e2e_s
    io_bytes = wl.prims.size * 8

    # stage-solve iteration counts of the benchmark workload: one more step
    # with the device histograms on, after all timing (counting uses atomics)
    e2e_sim.set_solver_stats(True)
    e2e_sim.set_prims(pin)
    e2e_sim.step(wl.dt, 1)
    e2e_sim.check()
    hist = e2e_sim.solver_stats()
    e2e_sim.set_solver_stats(False)

    def _mean(h):
        n = sum(h.values())
        return sum(k * v for k, v in h.items()) / n if n else None
    solver = {"solves": sum(hist["fp64_passes"].values()),
              "fp32_iterations_mean": _mean(hist["fp32_iterations"]),
              "fp64_passes_mean": _mean(hist["fp64_passes"]),
              "fp32_iterations": {str(k): v for k, v in hist["fp32_iterations"].items()},
              "fp64_passes": {str(k): v for k, v in hist["fp64_passes"].items()},
              "converged_start": hist["starts"],
              "note": "one FP64 step of the benchmark workload, both implicit stages, counted after timing"}

    # roofline of the dominant kernel (FP64 form): FP64-pipe bound. Peak = the
    # FP64 FMA rate measured now on this GPU by the library's own probe
    # (independent FMA chains on every SM), x2 for FLOP/s; achieved = the
    # oracle-counted algorithmic flops of the kernel per cell x cells / its
    # CUDA-event time per launch
    hbm_gbs, peak_src, smax = _peaks()
    dom = max(kt64, key=lambda k: kt64[k][0])
    dom_ms, dom_n = kt64[dom]
    per_launch_ms = dom_ms / dom_n
    fma_rate, n_sm = fp64_fma_rate(f"cuda:{local}")
    fp64_peak = 2.0 * fma_rate / 1e12
    alg = ALG_FP64_FLOPS_PER_CELL.get(dom)
    achieved = alg * wl.cells / (per_launch_ms * 1e-3) / 1e12 if alg else None
    issued = FP64_INST_PER_CELL[dom] * wl.cells / (per_launch_ms * 1e-3)
    hbm_achieved = BYTES_PER_CELL[dom] * wl.cells / (per_launch_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "achieved": achieved, "peak": fp64_peak, "unit": "TFLOP/s",
                "frac": achieved / fp64_peak if achieved else None,
                "traffic": DRAM_BYTES_PER_CELL[dom] * wl.cells, "kernel": dom,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per cell on the 512^2 "
                                  "step, times the cells of this launch",
                "kernel_ms_per_launch": per_launch_ms,
                "peak_source": f"measured: FP64 FMA chains on all {n_sm} SMs, CUDA events (rmhd_fp64_fma_rate), x2",
                "alg_flops_per_cell": alg,
                "fp64_inst_per_cell": FP64_INST_PER_CELL[dom],
                "issue_frac": issued / fma_rate,
                "hbm_gbs": hbm_achieved, "hbm_frac": hbm_achieved / hbm_gbs,
                "hbm_peak_gbs": hbm_gbs, "hbm_peak_source": peak_src}
    step_bytes = 1056.0  # algorithmic HBM bytes per cell-update of the whole step
    kernels = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1]} for k, v in kt64.items()}
    kernels_mx = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1]} for k, v in ktmx.items()}
    kernels_ff = {k: {"ms_per_launch": v[0] / max(v[1], 1), "launches": v[1]} for k, v in ktff.items()}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline()

    if rank == 0:
        # verbose sections first; the standard keys and a compact summary of
        # every form and workload at the end of the line
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K, "warmup": W,
                "ms_per_step": ms64 / K, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic",
                "config": {"workload": workload_name(args.n), "cells_per_gpu": wl.cells,
                           "parallelism": (f"slabs along y x{world}, NCCL halo exchange" if decomposed
                                           else f"replicas x{world}"),
                           "l2": "inputs larger than L2: state+workspace %.2f GB > 129 MB" %
                                 (sim64.workspace.numel() / 1e9)},
                "other_workloads": extra,
                "batch": batch,
                "adjoint": adjoint,
                "solver_stats": solver,
                "kernels": kernels,
                "mixed": {"value": value_mx, "ms_per_step": msmx / K, "dtype": "f32 flux / f64 source",
                          "rel_l1_vs_fp64": rel_l1_mixed, "speedup_vs_fp64": value_mx / value, "kernels": kernels_mx},
                "floatfloat": {"value": value_ff, "ms_per_step": msff / K, "dtype": "f32x2 flux / f64 source",
                               "rel_linf_vs_fp64": rel_linf_ff, "rel_l1_vs_fp64": rel_l1_ff,
                               "speedup_vs_fp64": value_ff / value, "kernels": kernels_ff},
                "hbm_roofline_step": {"bytes_per_cell_update": step_bytes,
                                      "achieved_gbs": step_bytes * value / world / 1e9,
                                      "frac": step_bytes * value / world / 1e9 / hbm_gbs},
                "cpu_baseline": cpu,
                "clocks": clocks,
                "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": io_bytes,
                        "d2h_bytes_per_step": io_bytes},
                "gpu_launches": 4 * K,
                "roofline": roofline}
        summ = {"fp64": round(value / 1e6, 1), "mixed": round(value_mx / 1e6, 1),
                "mixed_speedup": round(value_mx / value, 2), "mixed_rel_l1": float(f"{rel_l1_mixed:.2e}"),
                "ff": round(value_ff / 1e6, 1), "ff_rel_linf": float(f"{rel_linf_ff:.2e}")}
        if extra:
            tfx = extra["two_fluid_512"]
            summ.update({"tf512_fp64": round(tfx["fp64"] / 1e6, 1), "tf512_mixed": round(tfx["mixed"] / 1e6, 1),
                         "ssp3_fp64": round(extra["khi_1024_ssp3"]["fp64"] / 1e6, 1),
                         "khi3d_fp64": round(extra["khi3d_128"]["fp64"] / 1e6, 1)})
        if batch:
            summ.update({"batch_mixed": round(batch["value"] / 1e6, 1),
                         "batch_rel_l1": float(f"{batch['rel_l1_mixed_vs_fp64_max_over_tubes']:.2e}")})
        if adjoint:
            summ.update({"adjoint_over_fwd": round(adjoint["adjoint_over_fwd"], 2),
                         "tf_adjoint_over_fwd": round(adjoint["two_fluid"]["adjoint_over_fwd"], 2)})
        summ.update({"alu_frac": round(roofline["frac"], 3) if roofline["frac"] else None,
                     "hbm_frac_kernel": round(roofline["hbm_frac"], 4)})
        line["summary_Mcell_updates_per_s"] = summ
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
