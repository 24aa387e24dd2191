"""CUDA path (through the C ABI) against the FP64 CPU oracle.

Tolerances (written here, derived in the design notes):
  * FP64 fields: relative max-norm 1e-12 for w; wdot is compared on the scale
    of the state, max|dt * (wdot_gpu - wdot_oracle)| / max|w| < 1e-12 (wdot is
    a small difference of terms of size g w, so its own relative error carries
    the cancellation of the moment sum; the bound 1e-10 on its plain relative
    max-norm is also checked);
  * FP32 fields: relative max-norm 1e-5 (w) and the same state-scale rule for
    wdot, on runs of up to 2000 steps;
  * cut masks and crack-tip positions: bit-exact (FP64); the tip on the 2^-32
    dh grid, exact where the oracle's decision margin exceeds the rounding;
  * K history: within 1e-9 of max|K| in FP64 and 0.5 % of max|K| in FP32.
"""
import math

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


def _tol(storage):
    return 1e-12 if storage == "f64" else 1e-5


def run_pair(oracle_mod, lbm, problem, storage, steps, init=None, chunks=None):
    o = oracle_mod.Oracle(problem)
    g = lbm.Lattice(problem, storage)
    if init is not None:
        o.set_fields(*init)
        g.set_fields(*init)
    for n in (chunks or [steps]):
        o.step(n)
        g.step(n)
    return o, g


def compare_fields(o, g, storage, dt=1.0, wdot_rel=None):
    w_o, wd_o = o.fields()
    w_g, wd_g = g.fields()
    scale = max(np.abs(w_o).max(), 1e-300)
    ew = np.abs(w_g - w_o).max() / scale
    ewd = np.abs(wd_g - wd_o).max() * dt / scale
    tol = _tol(storage)
    assert ew < tol, f"w rel err {ew:.3e}"
    assert ewd < tol, f"wdot state-scale err {ewd:.3e}"
    if wdot_rel is not None:
        e = np.abs(wd_g - wd_o).max() / max(np.abs(wd_o).max(), 1e-300)
        assert e < wdot_rel, f"wdot rel err {e:.3e}"
    return ew, ewd


def compare_masks(o, g):
    ch, cv = o.cuts()
    assert np.array_equal(g.cut_mask("h"), ch.astype(bool))
    assert np.array_equal(g.cut_mask("v"), cv.astype(bool))


def compare_crack(o, g, storage, exact_tip=True):
    co = o.crack()
    cg = g.crack_state()
    ho = o.history()
    hg = g.history()
    assert cg["step"] == co["step"]
    n = len(ho["K"])
    assert len(hg["K"]) == n
    if n == 0:
        return
    Kscale = max(np.abs(ho["K"]).max(), 1e-300)
    ktol = 1e-9 if storage == "f64" else 5e-3
    assert np.abs(hg["K"] - ho["K"]).max() < ktol * Kscale
    assert np.array_equal(hg["npairs"], ho["npairs"])
    if exact_tip:
        assert cg["tip_q"] == co["tip_q"]
        assert np.array_equal(hg["tip_q"], ho["tip_q"])
        assert np.array_equal(hg["v"] == 0, ho["v"] == 0)


# ----------------------------------------------------------------- cases

@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_plain_128_stationary_2000_steps(oracle_mod, gpu, storage, bc_mode):
    """128x128, crack to x = 32 on y = 64, +-1e-3 ramped over 200 steps, 2000 steps."""
    p = W.plain_fp64(bc_mode)
    o, g = run_pair(oracle_mod, gpu, p, storage, W.PLAIN_FP64_STEPS, chunks=[1, 63, 64, 1872])
    compare_fields(o, g, storage, wdot_rel=1e-10 if storage == "f64" else None)
    compare_masks(o, g)
    compare_crack(o, g, storage)


def _mixed_problem(bc_mode, nx=37, ny=29):
    p = W.base_problem(nx, ny, bc_mode=bc_mode, edges=("free", "dirichlet", "dirichlet", "free"))
    # (with macroscopic faces a ligament of one column at the free left edge
    # or of two at the Dirichlet right edge is unstable and rejected at
    # create: start the crack at the edge and stop it three columns short of
    # the right edge on lattices too narrow for wider ligaments)
    x_start = min(4.3, 0.2 * nx) if 0.2 * nx >= 1.5 else 0.0
    x_tip = nx * 0.55 if nx >= 10 else nx - 3.3
    p = W.with_crack(p, mode="stationary", y=float(ny // 2), x_start=x_start, x_tip=x_tip)
    p["loads"] = [{"edge": "right", "kind": "const", "amp": 3e-4, "t": 0.0},
                  {"edge": "bottom", "kind": "sin2", "amp": -5e-4, "t": 40.0}]
    return p


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
@pytest.mark.parametrize("shape", [(37, 29), (130, 70), (5, 9), (257, 33)])
def test_ragged_mixed_edges_random_state(oracle_mod, gpu, storage, bc_mode, shape):
    nx, ny = shape
    p = _mixed_problem(bc_mode, nx, ny)
    init = W.random_state(nx, ny, seed=nx * 1000 + ny, dtype=np.float32 if storage == "f32" else np.float64)
    o, g = run_pair(oracle_mod, gpu, p, storage, 300, init=init, chunks=[1, 2, 64, 233])
    compare_fields(o, g, storage)
    compare_masks(o, g)
    compare_crack(o, g, storage)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_periodic_lattice(oracle_mod, gpu, storage):
    p = W.base_problem(50, 34, edges=("periodic",) * 4)
    init = W.random_state(50, 34, seed=4, dtype=np.float32 if storage == "f32" else np.float64)
    o, g = run_pair(oracle_mod, gpu, p, storage, 400, init=init, chunks=[1, 399])
    compare_fields(o, g, storage)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_periodic_x_dirichlet_y(oracle_mod, gpu, storage):
    p = W.base_problem(64, 30, bc_mode="bounceback", edges=("periodic", "periodic", "dirichlet", "dirichlet"))
    p = W.with_crack(p, mode="stationary", y=15.0, x_start=10.0, x_tip=40.0)
    p = W.with_antisymmetric_ramp(p, 1e-3, 50.0)
    o, g = run_pair(oracle_mod, gpu, p, storage, 300, chunks=[300])
    compare_fields(o, g, storage)
    compare_crack(o, g, storage)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_prescribed_growth_to_clamp(oracle_mod, gpu, storage, bc_mode):
    p = W.prescribed_strip(96, 48, 0.6, bc_mode=bc_mode, crack_len=20.0, r_min=2.25)
    o, g = run_pair(oracle_mod, gpu, p, storage, 300, chunks=[7, 64, 229])
    compare_fields(o, g, storage)
    compare_masks(o, g)
    compare_crack(o, g, storage)
    assert g.crack_state()["flags"] & 1


def test_kcrit_growth_fp64(oracle_mod, gpu):
    p = W.base_problem(96, 48, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_tip=20.0, K_C=K_C, v_max=0.85, r0=2.0)
    o, g = run_pair(oracle_mod, gpu, p, "f64", 400, chunks=[400])
    compare_fields(o, g, "f64")
    compare_masks(o, g)
    # decisions are bit-exact when |K| is not within rounding of K_C
    ho = o.history()
    margin = np.min(np.abs(np.abs(ho["K"][ho["npairs"] > 0]) / K_C - 1.0))
    compare_crack(o, g, "f64", exact_tip=margin > 1e-9)
    assert (ho["v"] > 0).sum() > 10


def test_kcrit_growth_fp32_tolerance(oracle_mod, gpu):
    """FP32 fields with an FP64 K decision: the tip trajectory follows the
    oracle's within one lattice spacing and the growth count within a few steps."""
    p = W.base_problem(96, 48, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_tip=20.0, K_C=K_C, v_max=0.85, r0=2.0)
    o, g = run_pair(oracle_mod, gpu, p, "f32", 300, chunks=[300])
    ho, hg = o.history(), g.history()
    assert np.abs(hg["tip_q"] - ho["tip_q"]).max() < 2**32
    assert abs(int((hg["v"] > 0).sum()) - int((ho["v"] > 0).sum())) <= 3


def test_full_size_kcrit_grid_random_state(oracle_mod, gpu):
    """4096 x 2048 FP32 in the launch shape the benchmark times: every output
    after 12 steps from a seeded state, against the oracle at full size."""
    p = W.kcrit_single()
    init = W.random_state(p["nx"], p["ny"], seed=21, dtype=np.float32)
    o, g = run_pair(oracle_mod, gpu, p, "f32", 12, init=init, chunks=[12])
    compare_fields(o, g, "f32")
    compare_masks(o, g)
    compare_crack(o, g, "f32")


# -------------------------------------------------------- path equivalence

def test_graph_replay_equals_single_steps(gpu):
    p = W.plain_fp64("macroscopic")
    a = gpu.Lattice(p, "f32")
    b = gpu.Lattice(p, "f32")
    a.step(130)
    for _ in range(130):
        b.step(1)
    wa, wda = a.fields()
    wb, wdb = b.fields()
    assert np.array_equal(wa, wb) and np.array_equal(wda, wdb)
    assert a.crack_state() == b.crack_state()


@pytest.mark.parametrize("rows", [1, 4, 7, 64, 300])
def test_launch_shape_does_not_change_results(gpu, rows):
    p = _mixed_problem("macroscopic", 130, 70)
    init = W.random_state(130, 70, seed=2, dtype=np.float32)
    a = gpu.Lattice(p, "f32")
    b = gpu.Lattice(p, "f32")
    a.set_fields(*init)
    b.set_fields(*init)
    b.set_launch(rows)
    a.step(100)
    b.step(100)
    assert np.array_equal(a.fields()[0], b.fields()[0])
    assert np.array_equal(a.fields()[1], b.fields()[1])


def test_cudamalloc_and_torch_allocator_agree(gpu):
    p = W.plain_fp64("bounceback")
    a = gpu.Lattice(p, "f64", torch_allocator=True)
    b = gpu.Lattice(p, "f64", torch_allocator=False)
    a.step(77)
    b.step(77)
    assert np.array_equal(a.fields()[0], b.fields()[0])


def test_device_fields_and_roundtrip(gpu):
    import torch
    p = _mixed_problem("macroscopic", 40, 30)
    g = gpu.Lattice(p, "f32")
    w0, wd0 = W.random_state(40, 30, seed=9, dtype=np.float32)
    g.set_fields(w0, wd0)
    w, wd = g.fields()
    assert np.array_equal(w, w0.astype(np.float32)) and np.array_equal(wd, wd0.astype(np.float32))
    g.step(0)
    g.step(5)
    wt, wdt = g.fields_device()
    torch.cuda.synchronize()
    w, wd = g.fields()
    assert np.array_equal(wt.cpu().numpy(), w) and np.array_equal(wdt.cpu().numpy(), wd)
    g2 = gpu.Lattice(p, "f32")
    g2.set_fields(torch.from_numpy(w).cuda(), torch.from_numpy(wd).cuda())
    assert np.array_equal(g2.fields()[0], w)


def test_nonfinite_state_is_reported(gpu):
    p = _mixed_problem("bounceback", 40, 30)
    g = gpu.Lattice(p, "f32")
    w = np.zeros((30, 40), np.float32)
    w[7, 9] = np.nan
    g.set_fields(w, np.zeros_like(w))
    g.step(3)
    with pytest.raises(gpu.LbmError) as ei:
        g.sync()
    assert ei.value.status == -4
    with pytest.raises(gpu.LbmError):
        g.step(1)
