"""The N > 1 paths without a GPU: the max-over-ranks reduction of bench.py on
a world_size-2 gloo group, the halo exchange schedule of the domain
decomposition along y (paper_1808_09721_gb300.slabs.exchange) on gloo groups of
2 and 3 ranks, periodic and outflow, and the reference arm (the CPU oracle)
launched under torchrun with 2 ranks, where rank 0 alone prints the JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        out[rank] = bench.reduce_max(1.5 + rank, world, "cpu")
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_reduce_max_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_under_torchrun_two_ranks():
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"


def _exchange_worker(rank, world, port, periodic, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_1808_09721_gb300.slabs import exchange, neighbours
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        n = 12
        # this rank's first rows (lo) and last rows (hi), tagged by rank and side
        send_lo = torch.arange(n, dtype=torch.float64) + 1000.0 * rank
        send_hi = torch.arange(n, dtype=torch.float64) + 1000.0 * rank + 500.0
        recv_lo = torch.full((n,), -1.0, dtype=torch.float64)
        recv_hi = torch.full((n,), -1.0, dtype=torch.float64)
        for r in exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic):
            r.wait()
        lo, hi = neighbours(rank, world, periodic)
        out[rank] = (lo, hi, recv_lo.tolist(), recv_hi.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic", [(2, True), (2, False), (3, True), (3, False)])
def test_halo_exchange_schedule_on_gloo(world, periodic):
    """Every slab receives its lower neighbour's last rows into its lower halo
    and its upper neighbour's first rows into its upper halo (cyclically when
    periodic; nothing at a global outflow boundary) -- also with two periodic
    ranks, where one peer is both neighbours."""
    import torch.multiprocessing as mp
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_exchange_worker, args=(world, _free_port(), periodic, out), nprocs=world, join=True)
    n = 12
    for rank in range(world):
        lo, hi, rlo, rhi = out[rank]
        if lo is None:
            assert rank == 0 and not periodic and rlo == [-1.0] * n
        else:
            assert lo == (rank - 1) % world
            assert rlo == [float(k) + 1000.0 * lo + 500.0 for k in range(n)]
        if hi is None:
            assert rank == world - 1 and not periodic and rhi == [-1.0] * n
        else:
            assert hi == (rank + 1) % world
            assert rhi == [float(k) + 1000.0 * hi for k in range(n)]


def test_neighbours_and_rows():
    from paper_1808_09721_gb300.slabs import neighbours, split_rows
    assert neighbours(0, 1, True) == (0, 0) and neighbours(0, 1, False) == (None, None)
    assert neighbours(0, 4, False) == (None, 1) and neighbours(3, 4, True) == (2, 0)
    assert split_rows(10, 3) == [4, 3, 3] and sum(split_rows(1024, 7)) == 1024
