"""Degenerate and boundary cases of the CUDA path against the oracle:
single-column and two-row lattices, a crack that starts with no severed
link, a tip exactly on a link, zero steps, and degenerate adjoint tapes."""
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


def _run(oracle_mod, lbm, p, storage, steps, seed=1):
    o = oracle_mod.Oracle(p)
    g = lbm.Lattice(p, storage)
    init = W.random_state(p["nx"], p["ny"], seed=seed, dtype=np.float64 if storage == "f64" else np.float32)
    o.set_fields(*init)
    g.set_fields(*init)
    o.step(steps)
    g.step(steps)
    return o, g


def _close(o, g, tol):
    wo, wdo = o.fields()
    wg, wdg = g.fields()
    scale = max(np.abs(wo).max(), 1e-300)
    assert np.abs(wg - wo).max() <= tol * scale
    assert np.abs(wdg - wdo).max() <= tol * scale


@pytest.mark.parametrize("edges", [("free", "free", "dirichlet", "dirichlet"), ("periodic", "periodic", "free", "dirichlet"),
                                   ("dirichlet", "dirichlet", "periodic", "periodic")])
@pytest.mark.parametrize("shape", [(1, 2), (1, 9), (3, 2), (2, 5)])
def test_tiny_lattices(oracle_mod, gpu, shape, edges):
    nx, ny = shape
    p = W.base_problem(nx, ny, edges=edges)
    p["loads"] = [{"edge": e, "kind": "sin2", "amp": 1e-3 * (k + 1), "t": 20.0}
                  for k, e in enumerate(("left", "right", "bottom", "top")) if edges[("left", "right", "bottom", "top").index(e)] == "dirichlet"]
    o, g = _run(oracle_mod, gpu, p, "f64", 150)
    _close(o, g, 1e-12)


@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_crack_that_starts_with_no_severed_link(oracle_mod, gpu, bc_mode):
    """x_start = x_tip between two link positions: nothing is severed at the
    start; prescribed growth then severs the links one by one."""
    p = W.base_problem(64, 24, bc_mode=bc_mode)
    p = W.with_crack(p, mode="prescribed", y=12.0, x_start=10.2, x_tip=10.2, v_rel=0.45)
    p = W.with_antisymmetric_ramp(p, 1e-3, 30.0)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f64")
    assert not g.cut_mask("v").any()
    o.step(120)
    g.step(120)
    _close(o, g, 1e-12)
    np.testing.assert_array_equal(g.cut_mask("v"), o.cuts()[1].astype(bool))
    assert g.crack_state()["tip_q"] == o.crack()["tip_q"]


@pytest.mark.parametrize("x_tip", [20.5, 21.0, 20.4999999])
def test_tip_on_and_next_to_a_link(oracle_mod, gpu, x_tip):
    """A link touching the tip is severed (closed segment): x_tip = 20.5 cuts
    column 20, 20.4999999 does not."""
    p = W.base_problem(48, 20, bc_mode="macroscopic")
    p = W.with_crack(p, mode="stationary", y=10.0, x_start=3.0, x_tip=x_tip)
    p = W.with_antisymmetric_ramp(p, 1e-3, 20.0)
    o, g = _run(oracle_mod, gpu, p, "f64", 80)
    np.testing.assert_array_equal(g.cut_mask("v"), o.cuts()[1].astype(bool))
    assert g.cut_mask("v")[9, 20] == (x_tip >= 20.5)
    _close(o, g, 1e-12)


def test_zero_steps_change_nothing(gpu):
    p = W.plain_fp64()
    g = gpu.Lattice(p, "f64")
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=4)
    g.set_fields(w0, wd0)
    g.step(0)
    w, wd = g.fields()
    np.testing.assert_array_equal(w, w0)
    np.testing.assert_array_equal(wd, wd0)
    assert g.crack_state()["step"] == 0


def test_adjoint_without_sensors_and_of_one_step(oracle_mod, gpu):
    p, _, w0, wd0, sens, tgt = W.adjoint_case("macro_growth", 1, seed=6)
    # no sensors: zero loss, zero gradient
    lat = gpu.Lattice(p, "f64")
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, np.zeros((0, 2), np.int32), 5)
    assert tape.forward(np.zeros((5, 0))) == 0.0
    dload, dw, dwd = tape.backward(device=False)
    assert not dload.any() and not dw.any() and not dwd.any()
    tape.close()
    # one step: the oracle's adjoint
    lat.reset()
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, 1)
    loss = tape.forward(tgt)
    dload, dw, dwd = tape.backward(device=False)
    ref = oracle_mod.adjoint(p, 1, sens, tgt, w0, wd0)
    assert loss == pytest.approx(ref["loss"], rel=1e-13)
    np.testing.assert_allclose(dload, ref["dload"], rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(dw, ref["dw0"], rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(dwd, ref["dwd0"], rtol=1e-12, atol=1e-20)
    tape.close()
    lat.close()
