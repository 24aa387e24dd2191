"""Two-tip cracks (both ends grow, Sec. 5.2) through the C ABI against the
oracle: tips and cut masks bit-exact, fields at the FP64/FP32 tolerances of
test_gpu_parity.py, K of both ends, and the same through the deferred crack
step, the adjoint, row slabs and batches."""
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


def _fields_close(o, g, tol):
    wo, wdo = o.fields()
    wg, wdg = g.fields()
    scale = max(np.abs(wo).max(), 1e-300)
    assert np.abs(wg - wo).max() <= tol * scale
    assert np.abs(wdg - wdo).max() <= tol * scale


def _ends_equal(o, g):
    ho, hl = o.history(), o.history_left()
    gr, gl = g.history(), g.history_left()
    np.testing.assert_array_equal(gr["tip_q"], ho["tip_q"])
    np.testing.assert_array_equal(gl["tip_q"], hl["tip_q"])
    np.testing.assert_array_equal(g.cut_mask("v"), o.cuts()[1].astype(bool))
    return ho, hl, gr, gl


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_prescribed_two_tips_across_column_blocks(oracle_mod, gpu, storage, bc_mode):
    """Both ends cross column-block boundaries (256 / 512 columns) and reach
    the far edges."""
    p = W.base_problem(700, 40, bc_mode=bc_mode)
    p = W.with_crack(p, mode="prescribed", y=20.0, x_start=300.3, x_tip=420.6, v_rel=0.6, two_tips=True)
    p = W.with_antisymmetric_ramp(p, 1e-3, 50.0)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, storage)
    for n in (7, 64, 700, 300):   # single launches and graph replay; both ends stop at the edges
        o.step(n)
        g.step(n)
    _fields_close(o, g, 1e-12 if storage == "f64" else 1e-5)
    _ends_equal(o, g)
    assert g.crack_state()["tip_q"] == 700 * 2**32 and g.crack_state_left()["tip_q"] == 0


@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_kcrit_centred_crack_fp64(oracle_mod, gpu, bc_mode):
    nx, ny = 160, 48
    p = W.base_problem(nx, ny, bc_mode=bc_mode)
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_start=62.0, x_tip=98.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f64")
    o.step(400)
    g.step(400)
    _fields_close(o, g, 1e-12)
    ho, hl, gr, gl = _ends_equal(o, g)
    for a, b in ((gr, ho), (gl, hl)):
        np.testing.assert_allclose(a["K"], b["K"], rtol=0, atol=1e-9 * np.abs(b["K"]).max())
        np.testing.assert_array_equal(a["npairs"], b["npairs"])
    assert (hl["v"] > 0).sum() > 10 and (ho["v"] > 0).sum() > 10


def test_kcrit_off_centre_fp32(oracle_mod, gpu):
    """FP32 fields with FP64 decisions: both ends follow the oracle within
    one lattice spacing."""
    p = W.base_problem(200, 48, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.45 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_start=50.0, x_tip=110.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32")
    o.step(350)
    g.step(350)
    for a, b in ((g.history(), o.history()), (g.history_left(), o.history_left())):
        assert np.abs(a["tip_q"] - b["tip_q"]).max() < 2**32
        assert abs(int((a["v"] > 0).sum()) - int((b["v"] > 0).sum())) <= 3


def test_deferred_crack_step_applies_both_ends(oracle_mod, gpu):
    """Reading the state between steps applies the pending crack step of both
    ends (one small kernel); the run stays bit-identical to an unread one."""
    p = W.base_problem(96, 32, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=16.0, x_start=40.2, x_tip=50.9, v_rel=0.45, two_tips=True)
    p = W.with_antisymmetric_ramp(p, 1e-3, 20.0)
    a = gpu.Lattice(p, "f64")
    b = gpu.Lattice(p, "f64")
    for _ in range(30):
        a.step(3)
        a.crack_state()
        a.crack_state_left()
    b.step(90)
    np.testing.assert_array_equal(a.fields()[0], b.fields()[0])
    assert a.crack_state() == b.crack_state() and a.crack_state_left() == b.crack_state_left()
    for k in ("K", "tip_q", "npairs"):
        np.testing.assert_array_equal(a.history_left()[k], b.history_left()[k])
    o = oracle_mod.Oracle(p)
    o.step(90)
    assert a.crack_state_left()["tip_q"] == o.left_tip_q()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_adjoint_with_two_tips(oracle_mod, gpu, storage):
    T = 150
    p = W.base_problem(300, 40, bc_mode="macroscopic", edges=("free", "free", "dirichlet", "dirichlet"))
    p = W.with_crack(p, mode="prescribed", y=20.0, x_start=120.4, x_tip=180.3, v_rel=0.7, two_tips=True)
    rng = np.random.default_rng(2)
    for e in ("bottom", "top"):
        p = W.with_series_load(p, e, 1e-3 * rng.standard_normal(T))
    dt = np.float64 if storage == "f64" else np.float32
    w0 = (1e-3 * rng.standard_normal((40, 300))).astype(dt).astype(np.float64)
    wd0 = (1e-4 * rng.standard_normal((40, 300))).astype(dt).astype(np.float64)
    sens = np.stack([rng.integers(0, 300, 10), rng.integers(0, 40, 10)], axis=1).astype(np.int32)
    tgt = 1e-3 * rng.standard_normal((T, 10))
    ref = oracle_mod.adjoint(p, T, sens, tgt, w0, wd0)
    lat = gpu.Lattice(p, storage)
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, T)
    loss = tape.forward(tgt)
    dload, dw, dwd = tape.backward(device=False)
    tol = 1e-10 if storage == "f64" else 1e-4
    assert loss == pytest.approx(ref["loss"], rel=1e-12 if storage == "f64" else 1e-4)
    for got, want in ((dload, ref["dload"]), (dw, ref["dw0"]), (dwd, ref["dwd0"])):
        assert np.abs(got - want).max() <= tol * np.abs(want).max()


def test_slabs_and_batches_with_two_tips(gpu):
    p = W.base_problem(300, 64, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 64.0)
    p = W.with_crack(p, mode="kcrit", y=32.0, x_start=110.0, x_tip=170.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    ref = gpu.Lattice(p, "f32")
    ref.step(250)
    dec = gpu.Decomp(p, 3, "f32")
    dec.step(250)
    np.testing.assert_array_equal(dec.fields()[0], ref.fields()[0])
    slab = dec.rank(dec.info()["crack_rank"])
    np.testing.assert_array_equal(slab.history_left()["tip_q"], ref.history_left()["tip_q"])
    dec.close()
    q = W.with_crack(p, mode="prescribed", y=32.0, x_start=100.0, x_tip=150.0, v_rel=0.3, two_tips=True)
    lats = [gpu.Lattice(p, "f32"), gpu.Lattice(q, "f32")]
    solo = [gpu.Lattice(p, "f32"), gpu.Lattice(q, "f32")]
    b = gpu.Batch(lats)
    b.step(200)
    for l, s in zip(lats, solo):
        s.step(200)
        np.testing.assert_array_equal(l.fields()[0], s.fields()[0])
        assert l.crack_state_left() == s.crack_state_left()
