"""Adjoint (include/lbm_adjoint.h) through the C ABI against the oracle's
adjoint, and its properties at full size.

Tolerances (written here, derived in the design notes):
  * FP64: the loss within 1e-12 relative; misfits within 1e-12 of max|w|;
    dL/dw*, dL/dw0 and dL/dwdot0 within 1e-10 relative max-norm (the CUDA
    adjoint transposes the moment form, the oracle the distribution form:
    the two round differently, over hundreds of steps);
  * FP32: loss within 1e-4 relative, misfits within 1e-5 of max|w|, the
    gradients within 1e-4 relative max-norm (FP32 adjoint fields, FP64 sums);
  * checkpointed and stored recordings: bit-identical;
  * directional derivatives against central differences of FP64 forward
    runs (exact for the quadratic misfit up to rounding): 1e-8 relative for
    the FP64 gradient, also on the 1024 x 1024, 8000-step problem; there the
    FP32 gradient agrees to 1e-4 of |grad| |d| per direction and to 1e-4 in
    max-norm with the FP64 gradient.
"""
import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KINDS_SMALL = ["macro_growth", "bb_growth", "bb_periodic", "all_dirichlet", "scaled_units", "no_crack"]
KINDS_WIDE = ["wide_macro", "wide_bb"]


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_12412_gb300 import lbm
    lbm.load_library()
    return lbm


def _relmax(a, b):
    return float(np.abs(np.asarray(a) - np.asarray(b)).max() / max(np.abs(np.asarray(b)).max(), 1e-300))


def gpu_adjoint(lbm, p, T, sens, tgt, w0, wd0, storage, every=0, band_rows=0):
    lat = lbm.Lattice(p, storage)
    if band_rows:
        lat.set_launch(band_rows)
    lat.set_fields(w0, wd0)
    tape = lbm.Tape(lat, sens, T, checkpoint_every=every)
    loss = tape.forward(tgt)
    mis = tape.misfits() if every == 0 else None
    dload, dw, dwd = tape.backward(device=False)
    tape.close()
    lat.close()
    return {"loss": loss, "misfits": mis, "dload": dload, "dw0": dw.astype(np.float64), "dwd0": dwd.astype(np.float64)}


def _tols(storage):
    if storage == "f64":
        return {"loss": 1e-12, "mis": 1e-12, "grad": 1e-10}
    return {"loss": 1e-4, "mis": 1e-5, "grad": 1e-4}


def _check_against_oracle(oracle_mod, lbm, kind, storage, T, band_rows=0, every=0):
    p, _, w0, wd0, sens, tgt = W.adjoint_case(kind, T, seed=21, ns=12 if kind.startswith("wide") else 6)
    if storage == "f32":
        w0 = w0.astype(np.float32).astype(np.float64)
        wd0 = wd0.astype(np.float32).astype(np.float64)
    ref = oracle_mod.adjoint(p, T, sens, tgt, w0, wd0)
    got = gpu_adjoint(lbm, p, T, sens, tgt, w0, wd0, storage, every=every, band_rows=band_rows)
    tol = _tols(storage)
    assert got["loss"] == pytest.approx(ref["loss"], rel=tol["loss"])
    if got["misfits"] is not None:
        scale = max(np.abs(ref["trace"]).max(), 1e-300)
        assert np.abs(got["misfits"] - (ref["trace"] - tgt)).max() <= tol["mis"] * scale
    for key in ("dload", "dw0", "dwd0"):
        err = _relmax(got[key], ref[key])
        assert err <= tol["grad"], f"{kind} {storage} {key}: rel err {err:.3e}"
    return got


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", KINDS_SMALL)
def test_adjoint_matches_oracle_small(oracle_mod, gpu, kind, storage):
    _check_against_oracle(oracle_mod, gpu, kind, storage, T=60)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", KINDS_WIDE)
def test_adjoint_matches_oracle_wide(oracle_mod, gpu, kind, storage):
    """Several column blocks with a ragged tail; the crack tip crosses a
    column-block boundary during the run."""
    _check_against_oracle(oracle_mod, gpu, kind, storage, T=300)


@pytest.mark.parametrize("band_rows", [1, 3, 7])
def test_adjoint_any_band_partition(oracle_mod, gpu, band_rows):
    """Short bands: the edge sums come from many CTAs, sensors fall into
    many bands."""
    _check_against_oracle(oracle_mod, gpu, "wide_macro", "f64", T=120, band_rows=band_rows)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("every", [1, 7, 64, 100])
def test_checkpointed_equals_stored(gpu, storage, every):
    """Recomputing segments from snapshots gives the same bits as keeping
    every misfit, and leaves the lattice where the forward run ended."""
    T = 250
    p, _, w0, wd0, sens, tgt = W.adjoint_case("wide_macro", T, seed=4, ns=9)
    a = gpu_adjoint(gpu, p, T, sens, tgt, w0, wd0, storage, every=0)
    lat = gpu.Lattice(p, storage)
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, T, checkpoint_every=every)
    loss = tape.forward(tgt)
    w_end, wd_end = lat.fields()
    st_end = lat.crack_state()
    dload, dw, dwd = tape.backward(device=False)
    w_after, wd_after = lat.fields()
    assert loss == a["loss"]
    np.testing.assert_array_equal(dload, a["dload"])
    np.testing.assert_array_equal(dw.astype(np.float64), a["dw0"])
    np.testing.assert_array_equal(dwd.astype(np.float64), a["dwd0"])
    np.testing.assert_array_equal(w_after, w_end)
    np.testing.assert_array_equal(wd_after, wd_end)
    assert lat.crack_state() == st_end
    # the lattice steps on from there exactly as an unrecorded run would
    lat.step(40)
    ref = gpu.Lattice(p, storage)
    ref.set_fields(w0, wd0)
    ref.step(T + 40)
    np.testing.assert_array_equal(lat.fields()[0], ref.fields()[0])
    tape.close()


def test_backward_twice_and_misfits(gpu, oracle_mod):
    T = 80
    p, _, w0, wd0, sens, tgt = W.adjoint_case("macro_growth", T, seed=9)
    lat = gpu.Lattice(p, "f64")
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, T)
    tape.forward(tgt)
    one = tape.backward(device=False)
    two = tape.backward(device=False)
    for x, y in zip(one, two):
        np.testing.assert_array_equal(x, y)
    ref = oracle_mod.adjoint(p, T, sens, tgt, w0, wd0, grad=False)
    np.testing.assert_allclose(tape.misfits(), ref["trace"] - tgt, rtol=0, atol=1e-12 * np.abs(ref["trace"]).max())


def _fd_check_fp64(gpu, p, loaded, T, sens, tgt, w0, wd0, n_dir, rel):
    """<grad, d> against central differences of GPU FP64 forward runs."""
    lat = gpu.Lattice(p, "f64")
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, T)
    tape.forward(tgt)
    dload, dw, dwd = tape.backward(device=False)
    series = {ld["edge"]: np.asarray(ld["series"]) for ld in p["loads"] if ld["kind"] == "series"}
    rng = np.random.default_rng(17)
    for _ in range(n_dir):
        du = {e: 1e-3 * rng.standard_normal(T) for e in loaded}
        dw_ = 1e-3 * rng.standard_normal(w0.shape)
        dwd_ = 1e-4 * rng.standard_normal(w0.shape)
        pred = float(np.sum(dw * dw_) + np.sum(dwd * dwd_))
        for e, d in du.items():
            pred += float(np.dot(dload[gpu.A.EDGE_INDEX[e]], d))
        Ls = []
        for sgn in (1.0, -1.0):
            lat.reset()
            for e, d in du.items():
                lat.set_loading(e, "series", series=series[e] + sgn * d)
            lat.set_fields(w0 + sgn * dw_, wd0 + sgn * dwd_)
            Ls.append(tape.forward(tgt))
        fd = (Ls[0] - Ls[1]) / 2.0
        assert fd == pytest.approx(pred, rel=rel)
    tape.close()


def test_fd_property_fp64_medium(gpu):
    T = 400
    p, loaded, w0, wd0, sens, tgt = W.adjoint_case("wide_macro", T, seed=12, ns=16)
    _fd_check_fp64(gpu, p, loaded, T, sens, tgt, w0, wd0, n_dir=4, rel=1e-8)


def test_reset_and_set_loading_reproduce_a_fresh_lattice(gpu):
    T = 130
    p, loaded, w0, wd0, sens, tgt = W.adjoint_case("wide_bb", T, seed=2)
    a = gpu.Lattice(p, "f32")
    a.set_fields(w0, wd0)
    a.step(77)
    a.reset()
    new = 2e-3 * np.random.default_rng(0).standard_normal(T)
    a.set_loading("bottom", "series", series=new)
    a.set_fields(w0, wd0)
    a.step(T)
    q = W.with_series_load(p, "bottom", new)
    b = gpu.Lattice(q, "f32")
    b.set_fields(w0, wd0)
    b.step(T)
    np.testing.assert_array_equal(a.fields()[0], b.fields()[0])
    np.testing.assert_array_equal(a.fields()[1], b.fields()[1])
    np.testing.assert_array_equal(a.cut_mask("v"), b.cut_mask("v"))
    assert a.crack_state() == b.crack_state()
    with pytest.raises(gpu.LbmError):
        a.set_loading("bottom", "series", series=np.zeros(T + 1))   # longer than at creation


def test_autograd_function(gpu):
    torch = pytest.importorskip("torch")
    T = 150
    p, _, w0, wd0, sens, tgt = W.adjoint_case("wide_macro", T, seed=5, ns=10)
    lat = gpu.Lattice(p, "f64")
    tape = gpu.Tape(lat, sens, T)
    top = next(ld["series"] for ld in p["loads"] if ld["edge"] == "top")
    u = torch.tensor(top, dtype=torch.float64, device="cuda", requires_grad=True)
    w0t = torch.tensor(w0, device="cuda", requires_grad=True)
    wd0t = torch.tensor(wd0, device="cuda", requires_grad=True)
    L = gpu.sensor_misfit(tape, "top", u, w0t, wd0t, tgt)
    (3.0 * L).backward()
    lat2 = gpu.Lattice(p, "f64")
    lat2.set_fields(w0, wd0)
    tape2 = gpu.Tape(lat2, sens, T)
    L2 = tape2.forward(tgt)
    dload, dw, dwd = tape2.backward(device=False)
    assert float(L.detach()) == pytest.approx(L2, rel=1e-13)
    np.testing.assert_allclose(u.grad.cpu().numpy(), 3.0 * dload[3], rtol=1e-12, atol=0)
    np.testing.assert_allclose(w0t.grad.cpu().numpy(), 3.0 * dw, rtol=1e-12, atol=0)
    np.testing.assert_allclose(wd0t.grad.cpu().numpy(), 3.0 * dwd, rtol=1e-12, atol=0)


def test_full_size_gradient_against_fp64_differences(gpu):
    """The 1024 x 1024, 8000-step sensor-misfit problem: the gradient of the
    top-edge history along 16 random unit directions against central
    differences (eps = 1e-3 |u|) of FP64 forward runs.  The FP64 adjoint
    agrees per direction to 1e-8; the FP32 one (FP32 forward and adjoint
    fields) to 1e-4 of |grad| |d| per direction and 1e-4 in max-norm against
    the FP64 gradient.  (Per direction and relative to <grad, d> itself the
    FP32 error reaches a few 1e-4 where <grad, d> is ten times below
    |grad| |d|.)"""
    a = W.adjoint_problem()
    p, T, sens = a["problem"], a["n_steps"], a["sensors"]
    # targets: the sensor trace of the reference history (FP64 run)
    ref = gpu.Lattice(W.with_series_load(p, "top", a["u_ref"]), "f64")
    tref = gpu.Tape(ref, sens, T)
    tref.forward(np.zeros((T, len(sens))))
    targets = tref.misfits()
    tref.close()
    ref.close()
    lat32 = gpu.Lattice(p, "f32")
    t32 = gpu.Tape(lat32, sens, T, checkpoint_every=int(round(np.sqrt(T))))
    t32.forward(targets)
    g32 = t32.backward(device=False)[0][3]
    lat64 = gpu.Lattice(p, "f64")
    t64 = gpu.Tape(lat64, sens, T)
    t64.forward(targets)
    g64 = t64.backward(device=False)[0][3]
    assert np.abs(g32 - g64).max() <= 1e-4 * np.abs(g64).max()
    gnorm = np.linalg.norm(g64)
    u = a["u_ctl"]
    eps = 1e-3 * np.linalg.norm(u)
    rng = np.random.default_rng(23)
    for _ in range(16):
        d = rng.standard_normal(T)
        d /= np.linalg.norm(d)
        Ls = []
        for sgn in (1.0, -1.0):
            lat64.reset()
            lat64.set_loading("top", "series", series=u + sgn * eps * d)
            Ls.append(t64.forward(targets))
        fd = (Ls[0] - Ls[1]) / (2.0 * eps)
        assert float(np.dot(g64, d)) == pytest.approx(fd, rel=1e-8)
        assert abs(float(np.dot(g32, d)) - fd) <= 1e-4 * gnorm
