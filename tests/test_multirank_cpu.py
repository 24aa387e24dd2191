"""The multi-rank (N > 1) paths on CPU, world size 2 over gloo: the
benchmark's replica timing (max over ranks, whole-job throughput), its
reference arm on a non-zero rank, and the row-slab split of a decomposed
lattice (host-only planning).  No GPU needed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench
from paper_2206_12412_gb300 import lbm


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.reduce_max(dist, times[rank], "cpu")
        v = bench.replica_value(world, 1000, 10, t)
        out.put((rank, t, v))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_replica_timing_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    times = [0.25, 0.5]
    mp.start_processes(_worker, args=(2, _free_port(), times, q), nprocs=2, join=True, start_method="spawn")
    got = sorted(q.get(timeout=60) for _ in range(2))
    for rank, t, v in got:
        assert t == 0.5                                 # the slowest rank sets the time
        assert v == pytest.approx(2 * 1000 * 10 / 0.5 / 1e9)   # both replicas' units


def test_reduce_max_without_process_group():
    assert bench.reduce_max(None, 3.5) == 3.5


def test_reference_arm_on_a_nonzero_rank_does_nothing(capsys):
    class Args:
        steps, warmup = 1, 3
    assert bench.run_reference(Args(), rank=1, world=2) == 0
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("ny,jc,hh,n", [(2048, 1024, 3, 4), (100, 50, 3, 2), (100, 26, 3, 4), (10, -1, 0, 5),
                                        (64, 32, 1, 8), (37, 18, 3, 3), (10, 5, 3, 3)])
def test_decomp_plan(ny, jc, hh, n):
    rs = lbm.lbm_decomp_plan(ny, jc, hh, n)
    assert rs[0] == 0 and rs[-1] == ny and len(rs) == n + 1
    assert all(b - a >= 2 for a, b in zip(rs, rs[1:]))
    if jc >= 0:   # each side's crack rows stay inside one slab (a boundary may be the crack line)
        assert not any(jc - hh < b < jc + hh and b != jc for b in rs[1:-1])
        below = [k for k, (a, b) in enumerate(zip(rs, rs[1:])) if a <= jc - hh and jc <= b]
        above = [k for k, (a, b) in enumerate(zip(rs, rs[1:])) if a <= jc and jc + hh <= b]
        assert len(below) == 1 and len(above) == 1
    even = [round(r * ny / n) for r in range(n + 1)]
    assert max(abs(a - b) for a, b in zip(rs, even)) <= max(hh, 1)


def test_decomp_plan_puts_a_near_boundary_on_the_crack_line():
    # an even boundary one row off the crack line goes onto it
    assert lbm.lbm_decomp_plan(100, 51, 3, 2) == [0, 51, 100]
    assert lbm.lbm_decomp_plan(100, 49, 3, 2) == [0, 49, 100]
    assert lbm.lbm_decomp_plan(100, 49, 1, 2) == [0, 50, 100]   # 50 is outside the rows 48, 49


def test_decomp_plan_rejects_impossible_splits():
    with pytest.raises(lbm.LbmError):
        lbm.lbm_decomp_plan(10, -1, 0, 6)        # slabs of fewer than 2 rows
    with pytest.raises(lbm.LbmError):
        lbm.lbm_decomp_plan(12, 6, 3, 5)         # the crack rows take 6 of 12 rows: five slabs cannot avoid them
