"""Row slabs as separate processes (lbm_slab_create / lbm_slab_export /
lbm_slab_import, include/lbm_decomp.h): two processes on the one GPU, each
owning one slab handle, exchange their boundary rows of w through host
buffers over a gloo process group after every step.  The slabs together are
bit-identical to the undivided lattice -- fields, and the crack state and
history on each slab that holds the crack -- also when the boundary is the
crack line itself, where both processes run the crack step and reach the
same K; and the run matches the FP64 oracle within the parity tolerances.
No kernel waits on another process: the exchange is on the host, between
steps."""
import os
import socket

import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_12412_gb300 import lbm
    lbm.load_library()
    return lbm


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem():
    p = W.base_problem(300, 96, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 96.0)
    return W.with_crack(p, mode="kcrit", y=48.0, x_tip=60.0, K_C=K_C, v_max=0.85, r0=2.0)


def _exchange(dist, torch, slab, rank, world):
    rows = torch.from_numpy(np.stack(slab.export_rows()))
    got = [torch.empty_like(rows) for _ in range(world)]
    dist.all_gather(got, rows)
    below = got[rank - 1][1].numpy() if rank > 0 else None        # the top row of the slab below
    above = got[rank + 1][0].numpy() if rank < world - 1 else None   # the bottom row of the slab above
    slab.import_rows(below, above)


def _worker(rank, world, port, row_start, storage, steps, seed, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        from paper_2206_12412_gb300 import lbm
        p = _problem()
        r0, r1 = row_start[rank], row_start[rank + 1]
        slab = lbm.Slab(p, r0, r1 - r0, storage)
        w0, wd0 = W.random_state(p["nx"], p["ny"], seed=seed, dtype=np.float64 if storage == "f64" else np.float32)
        slab.set_fields(w0[r0:r1], wd0[r0:r1])
        _exchange(dist, torch, slab, rank, world)
        for _ in range(steps):
            slab.step(1)
            _exchange(dist, torch, slab, rank, world)
        w, wd = slab.fields()
        cs = slab.crack_state()
        hist = slab.history()
        q.put((rank, w, wd, cs, hist))
        slab.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _run_ranks(row_start, storage, steps, seed):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = len(row_start) - 1
    pc = mp.start_processes(_worker, args=(world, _free_port(), row_start, storage, steps, seed, q), nprocs=world,
                            join=False, start_method="spawn")
    # take the results before joining: a child cannot exit while its queue
    # still holds data the parent has not read
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    while not pc.join(timeout=60):
        pass
    return res


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("row_start", [[0, 48, 96], [0, 60, 96]])
def test_two_processes_match_the_undivided_lattice_and_the_oracle(oracle_mod, gpu, storage, row_start):
    steps, seed = 160, 23
    res = _run_ranks(row_start, storage, steps, seed)
    p = _problem()
    ref = gpu.Lattice(p, storage)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=seed, dtype=np.float64 if storage == "f64" else np.float32)
    ref.set_fields(w0, wd0)
    ref.step(steps)
    w_ref, wd_ref = ref.fields()
    w = np.concatenate([r[1] for r in res])
    wd = np.concatenate([r[2] for r in res])
    np.testing.assert_array_equal(w, w_ref)
    np.testing.assert_array_equal(wd, wd_ref)
    cs_ref, h_ref = ref.crack_state(), ref.history()
    jc = 48
    holders = [r for r in res if row_start[r[0]] <= jc <= row_start[r[0] + 1]]
    assert len(holders) == (2 if jc in row_start else 1)
    for _, _, _, cs, hist in holders:       # one K and one crack state on every rank that holds the crack
        assert cs == cs_ref
        for k in h_ref:
            np.testing.assert_array_equal(hist[k], h_ref[k])
    assert (h_ref["v"] > 0).sum() > 5
    # and the oracle's undivided run
    o = oracle_mod.Oracle(p)
    o.set_fields(w0, wd0)
    o.step(steps)
    wo, _ = o.fields()
    tol = 1e-12 if storage == "f64" else 1e-5
    assert np.abs(w - wo).max() < tol * np.abs(wo).max()
    o.close()
    ref.close()
