"""The row-slab decomposition of the method on CPU: two gloo ranks each step
one slab of the lattice in the oracle (bottom / top edges of kind "halo"),
handing the post-collision values that cross their common boundary to each
other between the collision and the streaming -- the one exchange the
scheme needs per step -- and together reproduce the undivided oracle run bit
for bit: fields, severed links, the crack's tip and K history.  With the
crack rows inside one slab, K is formed there from whole site pairs (no sum
crosses ranks).  Also a lattice periodic in y, whose wrap-around joins the
last slab to the first.  On D2Q9 three values per column cross a boundary
(the axis and both diagonals), each read at its link's source column; a
diagonal that also leaves through a left or right edge keeps that edge's
rule, and across periodic left / right edges the source column wraps."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2206_12412_gb300 import workloads as W


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(kind):
    if kind == "kcrit":
        p = W.base_problem(120, 40, bc_mode="macroscopic")
        p = W.with_antisymmetric_ramp(p, 3e-3, 40.0)
        K_C = 0.5 * W.strip_reference_K(0.25, 3e-3, 40.0)
        return W.with_crack(p, mode="kcrit", y=26.0, x_tip=30.0, K_C=K_C, v_max=0.85, r0=2.0)
    if kind == "periodic":
        return W.base_problem(64, 30, edges=("free", "dirichlet", "periodic", "periodic"))
    if kind == "kcrit_d2q9":
        return dict(_problem("kcrit"), lattice="D2Q9")
    if kind == "periodic_d2q9":
        # periodic in x and y: diagonal sources wrap across the left / right
        # edges too
        return dict(W.base_problem(64, 30, edges=("periodic", "periodic", "periodic", "periodic")), lattice="D2Q9")
    if kind == "loaded_d2q9":
        # a Dirichlet left edge and a free right edge meet the slab boundary:
        # the corner diagonals take the left / right rules
        p = W.base_problem(48, 26, edges=("dirichlet", "free", "dirichlet", "dirichlet"))
        p = dict(p, lattice="D2Q9")
        p["loads"] = [{"edge": "left", "kind": "sin2", "amp": 1e-3, "t": 30.0},
                      {"edge": "bottom", "kind": "const", "amp": -5e-4, "t": 0.0},
                      {"edge": "top", "kind": "linear", "amp": 8e-4, "t": 40.0}]
        return p
    raise KeyError(kind)


def slab_problem(p, r0, r1):
    """Rows r0 .. r1 - 1 of p as a problem of its own with halo edges."""
    edges = list(p.get("edges", ("free", "free", "dirichlet", "dirichlet")))
    periodic = edges[2] == "periodic"
    if r0 > 0 or periodic:
        edges[2] = "halo"
    if r1 < p["ny"] or periodic:
        edges[3] = "halo"
    q = dict(p, ny=r1 - r0, edges=tuple(edges))
    q["loads"] = [ld for ld in p.get("loads", []) if not (ld["edge"] in ("bottom", "top")
                                                          and edges[2 if ld["edge"] == "bottom" else 3] == "halo")]
    cr = p.get("crack") or {"mode": "none"}
    if cr["mode"] != "none" and r0 < cr["y"] < r1:
        q["crack"] = dict(cr, y=cr["y"] - r0)
    else:
        q["crack"] = {"mode": "none"}
    return q


def _worker(rank, world, port, kind, row_start, steps, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        p = _problem(kind)
        r0, r1 = row_start[rank], row_start[rank + 1]
        sp = slab_problem(p, r0, r1)
        o = oracle.Oracle(sp)
        w0, wd0 = W.random_state(p["nx"], p["ny"], seed=9)
        o.set_fields(w0[r0:r1], wd0[r0:r1])
        below, above = sp["edges"][2] == "halo", sp["edges"][3] == "halo"
        for _ in range(steps):
            o.collide()
            rows = torch.from_numpy(np.stack([o.fs_row(0), o.fs_row(1)]))
            got = [torch.empty_like(rows) for _ in range(world)]
            dist.all_gather(got, rows)
            if below:   # what leaves the slab below across its top edge
                o.set_halo(0, got[(rank - 1) % world][1].numpy())
            if above:   # what leaves the slab above across its bottom edge
                o.set_halo(1, got[(rank + 1) % world][0].numpy())
            o.finish_step()
        w, wd = o.fields()
        ch, cv = o.cuts()
        cr = o.crack() if sp["crack"]["mode"] != "none" else None
        hist = o.history() if cr is not None else None
        q.put((rank, w, wd, cv, cr, hist))
        o.close()
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind,row_start", [("kcrit", [0, 14, 40]), ("kcrit", [0, 31, 40]), ("periodic", [0, 13, 30]),
                                            ("kcrit_d2q9", [0, 14, 40]), ("kcrit_d2q9", [0, 31, 40]),
                                            ("periodic_d2q9", [0, 13, 30]), ("loaded_d2q9", [0, 9, 26])])
def test_two_gloo_ranks_match_the_undivided_oracle(oracle_mod, kind, row_start):
    steps = 120
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = len(row_start) - 1
    pc = mp.start_processes(_worker, args=(world, _free_port(), kind, row_start, steps, q), nprocs=world,
                            join=False, start_method="spawn")
    # take the results before joining: a child cannot exit while its queue
    # still holds data the parent has not read
    res = sorted((q.get(timeout=120) for _ in range(world)), key=lambda t: t[0])
    while not pc.join(timeout=60):
        pass
    p = _problem(kind)
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=9)
    o.set_fields(w0, wd0)
    o.step(steps)
    w, wd = o.fields()
    np.testing.assert_array_equal(np.concatenate([r[1] for r in res]), w)
    np.testing.assert_array_equal(np.concatenate([r[2] for r in res]), wd)
    _, cv = o.cuts()
    np.testing.assert_array_equal(np.concatenate([r[3] for r in res]), cv)
    if kind.startswith("kcrit"):
        holder = [r for r in res if r[4] is not None]
        assert len(holder) == 1
        _, _, _, _, cr, hist = holder[0]
        co, ho = o.crack(), o.history()
        assert cr["tip_q"] == co["tip_q"] and cr["step"] == co["step"]
        for k in ho:
            np.testing.assert_array_equal(hist[k], ho[k])
        assert (ho["v"] > 0).sum() > 5
    o.close()


def test_halo_edges_are_bottom_and_top_only(oracle_mod):
    p = dict(_problem("periodic"), edges=("halo", "dirichlet", "periodic", "periodic"))
    with pytest.raises(ValueError):
        oracle_mod.Oracle(p)
