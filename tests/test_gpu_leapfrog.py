"""Leapfrog storage (LBM_F32_LEAPFROG): the state kept as the FP32 planes w_n
and w_{n-1} (Sec. 3, eq. integration makes wdot_n = (w_n - w_{n-1}) / dt),
12 bytes per site update.  Against the FP64 oracle within the FP32 parity
tolerance (1e-5 relative max-norm of w; wdot on the scale of the state), K
within 0.5 %, prescribed tips and masks exact; batches, row slabs,
checkpoints and the bulk-copy march bit-identical to the plain leapfrog
lattice; the calls that do not take it reject it."""
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


def _close(o, g, tol=1e-5, dt=1.0):
    wo, wdo = o.fields()
    wg, wdg = g.fields()
    scale = np.abs(wo).max()
    assert np.abs(wg - wo).max() < tol * scale, np.abs(wg - wo).max() / scale
    assert np.abs(wdg - wdo).max() * dt < tol * scale, np.abs(wdg - wdo).max() * dt / scale


def _same(a, b):
    for x, y in zip(a.fields(), b.fields()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.cut_mask("v"), b.cut_mask("v"))
    assert a.crack_state() == b.crack_state()
    ha, hb = a.history(), b.history()
    for k in ha:
        np.testing.assert_array_equal(ha[k], hb[k])


@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_plain_128_against_the_oracle(oracle_mod, gpu, bc_mode):
    p = W.plain_fp64(bc_mode)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32_lf")
    for n in (1, 63, 64, 1872):
        o.step(n)
        g.step(n)
    _close(o, g)
    ho, hg = o.history(), g.history()
    assert np.abs(hg["K"] - ho["K"]).max() < 5e-3 * np.abs(ho["K"]).max()
    np.testing.assert_array_equal(g.cut_mask("v"), o.cuts()[1].astype(bool))


def test_ragged_random_state_and_loaded_edges(oracle_mod, gpu):
    p = W.base_problem(261, 37, bc_mode="macroscopic", edges=("free", "dirichlet", "dirichlet", "free"))
    p = W.with_crack(p, mode="prescribed", y=18.0, x_start=4.3, x_tip=60.7, v_rel=0.5)
    p["loads"] = [{"edge": "right", "kind": "const", "amp": 3e-4, "t": 0.0},
                  {"edge": "bottom", "kind": "sin2", "amp": -5e-4, "t": 40.0}]
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32_lf")
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=4, dtype=np.float32)
    o.set_fields(w0, wd0)
    g.set_fields(w0, wd0)
    o.step(300)
    g.step(300)
    _close(o, g)
    np.testing.assert_array_equal(g.history()["tip_q"], o.history()["tip_q"])
    np.testing.assert_array_equal(g.cut_mask("v"), o.cuts()[1].astype(bool))


def test_full_size_benchmark_lattice(oracle_mod, gpu):
    p = W.kcrit_single()
    init = W.random_state(p["nx"], p["ny"], seed=21, dtype=np.float32)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32_lf")
    o.set_fields(*init)
    g.set_fields(*init)
    o.step(12)
    g.step(12)
    _close(o, g)


def test_kcrit_growth_and_the_edge_rule(oracle_mod, gpu):
    p = W.kcrit_centre_crack(scale=2)     # macroscopic rule on every boundary, both tips
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32_lf")
    o.step(1500)
    g.step(1500)
    ho, hg = o.history(), g.history()
    assert np.abs(hg["tip_q"] - ho["tip_q"]).max() < 2**32
    assert abs(int((hg["v"] > 0).sum()) - int((ho["v"] > 0).sum())) <= 3
    assert (ho["v"] > 0).sum() > 10


def test_batch_slabs_checkpoint_and_bulk_are_bit_identical(gpu, tmp_path):
    p = W.base_problem(2100, 230, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 50.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 230.0)
    p = W.with_crack(p, mode="kcrit", y=115.0, x_tip=300.0, K_C=K_C, v_max=0.85, r0=2.0)
    init = W.random_state(p["nx"], p["ny"], seed=8, dtype=np.float32)
    ref = gpu.Lattice(p, "f32_lf")
    ref.set_fields(*init)
    ref.step(130)
    # a batch of it and two other lattices
    others = W.batch_problems(2, seed=12)
    mem = [gpu.Lattice(q, "f32_lf") for q in [p] + others]
    mem[0].set_fields(*init)
    b = gpu.Batch(mem)
    b.set_shape(32, 16)
    b.step(130)
    b.close()
    _same(ref, mem[0])
    # row slabs, one boundary on the crack line
    d = gpu.Decomp(p, 3, "f32_lf", row_start=[0, 60, 115, 230])
    d.set_fields(*init)
    d.step(130)
    for x, y in zip(d.fields(), ref.fields()):
        np.testing.assert_array_equal(x, y)
    d.close()
    # the bulk-copy march
    c = gpu.Lattice(p, "f32_lf")
    c.set_bulk(True)
    c.set_fields(*init)
    c.step(130)
    _same(ref, c)
    # checkpoint and resume
    path = str(tmp_path / "lf.ckpt")
    c.save(path)
    e = gpu.Lattice(p, "f32_lf")
    e.load(path)
    c.step(70)
    e.step(70)
    _same(c, e)


def test_wdot_is_formed_from_the_two_planes(gpu):
    p = W.plain_fp64("macroscopic")
    g = gpu.Lattice(p, "f32_lf")
    rng = np.random.default_rng(2)
    w = (rng.standard_normal((128, 128)) * 1e-3).astype(np.float32)
    wd = (rng.standard_normal((128, 128)) * 1e-4).astype(np.float32)
    g.set_fields(w, wd)
    w2, wd2 = g.fields()
    np.testing.assert_array_equal(w2, w)
    # wdot = (w - (w - dt wdot)) / dt (dt = 1): the two roundings, of w - dt wdot
    # and of the difference, each at most half an ulp of |w| + |dt wdot|
    assert np.all(np.abs(wd2 - wd) <= 2.0 ** -23 * (np.abs(w) + np.abs(wd)) + 1e-30)


def test_rejected_where_not_built(gpu):
    with pytest.raises(gpu.LbmError):
        gpu.Lattice(dict(W.plain_fp64("bounceback"), lattice="D2Q9"), "f32_lf")
    with pytest.raises(gpu.LbmError):
        gpu.Lattice(W.kcrit_line(scale=8), "f32_lf")
    lat = gpu.Lattice(W.plain_fp64("macroscopic"), "f32_lf")
    with pytest.raises(gpu.LbmError):
        gpu.Tape(lat, np.array([[3, 3]]), 10)
