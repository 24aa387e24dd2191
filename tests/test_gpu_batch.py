"""Batched lattices: one kernel launch per step advances every lattice, and
each one ends bit-identical to the same lattice stepped alone (same kernel
arithmetic), with uneven sizes, crack modes and crack-face modes."""
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


def mixed_problems():
    ps = []
    ps.append(W.plain_fp64("macroscopic"))
    ps.append(W.plain_fp64("bounceback"))
    ps.append(W.prescribed_strip(96, 48, 0.6, crack_len=20.0, r_min=2.25))
    p = W.base_problem(96, 48, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
    ps.append(W.with_crack(p, mode="kcrit", y=24.0, x_tip=20.0,
                           K_C=0.5 * W.strip_reference_K(0.25, 2e-3, 48.0), v_max=0.85, r0=2.0))
    q = W.base_problem(37, 29, bc_mode="bounceback", edges=("free", "dirichlet", "dirichlet", "free"))
    q = W.with_crack(q, mode="stationary", y=14.0, x_start=4.3, x_tip=20.7)
    q["loads"] = [{"edge": "right", "kind": "const", "amp": 3e-4, "t": 0.0},
                  {"edge": "bottom", "kind": "sin2", "amp": -5e-4, "t": 40.0}]
    ps.append(q)
    ps.append(W.base_problem(50, 34, edges=("periodic",) * 4))
    ps.extend(W.batch_problems(6, seed=11))
    return ps


def _same(a, b):
    wa, wda = a.fields()
    wb, wdb = b.fields()
    assert np.array_equal(wa, wb) and np.array_equal(wda, wdb)
    assert np.array_equal(a.cut_mask("v"), b.cut_mask("v"))
    sa, sb = a.crack_state(), b.crack_state()
    assert sa == sb
    ha, hb = a.history(), b.history()
    for k in ha:
        assert np.array_equal(ha[k], hb[k])


@pytest.mark.parametrize("storage", ["f32", "f64", "f32_f16"])
@pytest.mark.parametrize("band_rows", [0, 5])
def test_batch_equals_solo_runs(gpu, storage, band_rows):
    ps = mixed_problems()
    solo = [gpu.Lattice(p, storage) for p in ps]
    mem = [gpu.Lattice(p, storage) for p in ps]
    for p, s, m in zip(ps, solo, mem):
        if p["crack"]["mode"] == "none":
            init = W.random_state(p["nx"], p["ny"], seed=7, dtype=np.float64 if storage == "f64" else np.float32)
            s.set_fields(*init)
            m.set_fields(*init)
    b = gpu.Batch(mem, band_rows=band_rows)
    assert b.info()["lattices"] == len(ps)
    b.step(1)
    b.step(150)
    for s in solo:
        s.step(151)
    for s, m in zip(solo, mem):
        _same(s, m)
    b.close()


def test_batch_then_solo_steps_continue(gpu):
    ps = W.batch_problems(4, seed=5)
    solo = [gpu.Lattice(p, "f32") for p in ps]
    mem = [gpu.Lattice(p, "f32") for p in ps]
    b = gpu.Batch(mem)
    b.step(70)
    b.close()
    for m in mem:
        m.step(30)
    for s in solo:
        s.step(100)
    for s, m in zip(solo, mem):
        _same(s, m)


def test_batch_rejects_mixed_storage_and_diverged_steps(gpu):
    ps = W.batch_problems(2, seed=6)
    a = gpu.Lattice(ps[0], "f32")
    c = gpu.Lattice(ps[1], "f64")
    with pytest.raises(gpu.LbmError):
        gpu.Batch([a, c])
    d = gpu.Lattice(ps[1], "f32")
    b = gpu.Batch([a, d])
    a.step(1)
    with pytest.raises(gpu.LbmError) as ei:
        b.step(1)
    assert ei.value.status == -6
    b.close()


# ------------------------------------------------ batched path vs the oracle

def oracle_batch_problems():
    """Eight uneven lattices the oracle steps in seconds: K-criterion and
    prescribed growth, macroscopic and bounce-back crack faces, ragged widths
    (one lattice spans two column blocks) and seeded loads."""
    rng = np.random.default_rng(41)
    shapes = [(64, 32), (97, 45), (128, 64), (160, 96), (192, 128), (256, 64), (221, 101), (600, 48)]
    ps = []
    for q, (nx, ny) in enumerate(shapes):
        bc = "macroscopic" if q % 2 == 0 else "bounceback"
        u0 = float(np.exp(rng.uniform(np.log(1e-3), np.log(3e-3))))
        p = W.base_problem(nx, ny, bc_mode=bc)
        p = W.with_antisymmetric_ramp(p, u0, 100.0)
        length = float(rng.uniform(0.15, 0.35)) * nx
        if q % 4 < 2:
            K_C = W.strip_reference_K(0.25, u0, float(ny)) * float(rng.uniform(0.4, 0.6))
            p = W.with_crack(p, mode="kcrit", y=float(ny // 2), x_tip=length, K_C=K_C, v_max=0.85, r0=2.0)
        else:
            p = W.with_crack(p, mode="prescribed", y=float(ny // 2), x_tip=length,
                             v_rel=float(rng.uniform(0.1, 0.7)))
        p["hist_cap"] = 4096
        ps.append(p)
    return ps


@pytest.mark.parametrize("storage,rows", [("f64", 16), ("f32", 16), ("f32", -1)])
def test_batch_matches_the_oracle(oracle_mod, gpu, storage, rows):
    """Every lattice of one batch (one launch per step for all eight) against
    the FP64 oracle on the same problem, element by element: fields within
    1e-12 (FP64) / 1e-5 (FP32) relative max-norm (wdot on the scale of the
    state), cut masks and tips bit-exact in FP64 where the oracle's K
    decision margin exceeds 1e-9, K within 1e-9 / 0.5 % of max|K|; in FP32
    the K-criterion tips within one spacing and the growth count within 3.
    Bands of 16 rows, and the balanced step (rows = -1) in FP32."""
    from test_gpu_parity import compare_crack, compare_fields, compare_masks
    ps = oracle_batch_problems()
    steps = 400
    lats = [gpu.Lattice(p, storage) for p in ps]
    b = gpu.Batch(lats, band_rows=rows)
    b.step(1)
    b.step(steps - 1)
    b.close()
    grew = 0
    for p, g in zip(ps, lats):
        o = oracle_mod.Oracle(p)
        o.step(steps)
        compare_fields(o, g, storage)
        ho, hg = o.history(), g.history()
        kc = p["crack"]["mode"] == "kcrit"
        grew += int((ho["v"] > 0).sum() > 0)
        if storage == "f64":
            compare_masks(o, g)
            exact = True
            if kc and (ho["npairs"] > 0).any():
                margin = np.min(np.abs(np.abs(ho["K"][ho["npairs"] > 0]) / p["crack"]["K_C"] - 1.0))
                exact = margin > 1e-9
            compare_crack(o, g, storage, exact_tip=exact)
        elif kc:
            assert np.abs(hg["tip_q"] - ho["tip_q"]).max() < 2**32
            assert abs(int((hg["v"] > 0).sum()) - int((ho["v"] > 0).sum())) <= 3
        else:
            compare_masks(o, g)
            compare_crack(o, g, storage)
        o.close()
        g.close()
    assert grew >= 6   # the cracks of most lattices moved within the run


# ------------------------------------------------------ launch shapes, tuner

@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("threads,rows", [(32, 8), (64, 5), (32, 64), (128, 32), (32, 0), (128, 0),
                                          (32, -1), (64, -1), (128, -1), (64, -2), (128, -2)])
def test_every_launch_shape_gives_the_solo_bits(gpu, storage, threads, rows):
    """CTAs of 32, 64 or 128 threads over bands of any height, and the
    balanced step (rows = -1: runs of row pieces, several lattices per CTA,
    a lattice with the macroscopic rule on its outer edges among them): each
    lattice of the batch still ends bit-identical to its solo run (graph
    chunks and single launches)."""
    ps = mixed_problems() + [W.kcrit_centre_crack(scale=2)]
    solo = [gpu.Lattice(p, storage) for p in ps]
    mem = [gpu.Lattice(p, storage) for p in ps]
    for p, s, m in zip(ps, solo, mem):
        if p["crack"]["mode"] == "none":
            init = W.random_state(p["nx"], p["ny"], seed=9, dtype=np.float64 if storage == "f64" else np.float32)
            s.set_fields(*init)
            m.set_fields(*init)
    b = gpu.Batch(mem)
    b.set_shape(threads, rows)
    info = b.info()
    assert (info["threads"], info["band_rows"]) == (threads, rows)
    b.step(3)
    b.step(130)
    for s in solo:
        s.step(133)
    for s, m in zip(solo, mem):
        _same(s, m)
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f64", "f32_bf16", "f32_f16", "f32_lf"])
@pytest.mark.parametrize("threads,rows", [(32, 1), (64, 2), (128, 3), (32, 16), (128, 0), (64, -1)])
def test_two_row_lookahead_gives_the_solo_bits(gpu, storage, threads, rows):
    """The march with two rows of loads in flight (and bands of 1, 2 or 3
    rows, where the lookahead runs past the band) is the same arithmetic:
    each lattice ends bit-identical to its solo run."""
    ps = mixed_problems()
    solo = [gpu.Lattice(p, storage) for p in ps]
    mem = [gpu.Lattice(p, storage) for p in ps]
    for p, s, m in zip(ps, solo, mem):
        if p["crack"]["mode"] == "none":
            init = W.random_state(p["nx"], p["ny"], seed=21, dtype=np.float64 if storage == "f64" else np.float32)
            s.set_fields(*init)
            m.set_fields(*init)
    b = gpu.Batch(mem)
    b.set_shape(threads, rows)
    b.set_lookahead(2)
    info = b.info()
    assert (info["threads"], info["band_rows"], info["lookahead"]) == (threads, rows, 2)
    b.step(3)
    b.step(130)
    b.set_lookahead(1)
    b.step(7)
    for s in solo:
        s.step(140)
    for s, m in zip(solo, mem):
        _same(s, m)
    b.close()


def test_tune_leaves_the_lattices_as_they_were_and_caches_the_shape(gpu):
    ps = W.batch_problems(12, seed=8)
    solo = [gpu.Lattice(p, "f32") for p in ps]
    mem = [gpu.Lattice(p, "f32") for p in ps]
    b = gpu.Batch(mem)
    b.step(37)                       # a pending crack step at the tuning call
    r = b.tune(trial_steps=6)
    assert r["threads"] in (32, 64, 128) and r["band_rows"] in (-2, -1, 0, 8, 16, 32, 64) and r["lookahead"] in (1, 2)
    assert not r["from_cache"] and r["us_per_step"] > 0
    info = b.info()
    assert (info["threads"], info["band_rows"], info["lookahead"]) == (r["threads"], r["band_rows"], r["lookahead"])
    b.step(63)
    for s in solo:
        s.step(100)
    for s, m in zip(solo, mem):
        _same(s, m)                  # the trials left no trace
    b.close()
    # a second batch of the same lattices takes the cached shape
    mem2 = [gpu.Lattice(p, "f32") for p in ps]
    b2 = gpu.Batch(mem2)
    r2 = b2.tune(trial_steps=6)
    assert r2["from_cache"] and (r2["threads"], r2["band_rows"], r2["lookahead"]) == \
        (r["threads"], r["band_rows"], r["lookahead"])
    b2.close()


def test_shape_arguments_are_checked(gpu):
    ps = W.batch_problems(2, seed=6)
    lats = [gpu.Lattice(p, "f32") for p in ps]
    b = gpu.Batch(lats)
    for t, r in ((48, 16), (256, 16), (32, -3)):
        with pytest.raises(gpu.LbmError) as ei:
            b.set_shape(t, r)
        assert ei.value.status == -1
    for la in (0, 3):
        with pytest.raises(gpu.LbmError) as ei:
            b.set_lookahead(la)
        assert ei.value.status == -1
    with pytest.raises(gpu.LbmError):
        b.tune(trial_steps=1)
    b.close()


# ----------------------------------------------------- persistent batched form

@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("threads,rows", [(128, 16), (32, 32), (64, -1)])
def test_persistent_launch_gives_the_solo_bits(gpu, storage, threads, rows):
    """One cooperative launch for many steps (grid barrier between steps),
    including a lattice with the macroscopic rule on its outer edges (its
    edge-rule units after a second barrier): bit-identical to solo runs."""
    ps = mixed_problems()[:6] + [W.kcrit_centre_crack(scale=2)]
    solo = [gpu.Lattice(p, storage) for p in ps]
    mem = [gpu.Lattice(p, storage) for p in ps]
    for p, s, m in zip(ps, solo, mem):
        if p["crack"]["mode"] == "none":
            init = W.random_state(p["nx"], p["ny"], seed=13, dtype=np.float64 if storage == "f64" else np.float32)
            s.set_fields(*init)
            m.set_fields(*init)
    b = gpu.Batch(mem)
    b.set_shape(threads, rows)
    b.set_persistent(True)
    b.step(1)
    b.step(150)
    b.set_persistent(False)
    b.step(64)                       # and back to per-step launches
    for s in solo:
        s.step(215)
    for s, m in zip(solo, mem):
        _same(s, m)
    b.close()


def test_bounded_barrier_wait_gives_up_with_a_timeout(gpu):
    """A barrier that expects more CTAs than were launched is never
    completed: every wait gives up after its budget and the call returns
    LBM_ERR_TIMEOUT; a barrier that all its CTAs reach completes."""
    import torch
    s = torch.cuda.current_stream().cuda_stream
    gpu.lbm_barrier_probe(4, 4, 1 << 24, s)
    gpu.lbm_barrier_probe(1, 1, 1000, s)
    with pytest.raises(gpu.LbmError) as ei:
        gpu.lbm_barrier_probe(1, 2, 200000, s)
    assert ei.value.status == -5
    with pytest.raises(gpu.LbmError) as ei:
        gpu.lbm_barrier_probe(3, 8, 200000, s)
    assert ei.value.status == -5
    gpu.lbm_barrier_probe(2, 2, 1 << 24, s)   # the device is still usable
