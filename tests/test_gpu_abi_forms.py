"""The call forms of the C ABI that take the state in other shapes:
strided field copies (lbm_fields_strided / lbm_set_fields_strided), a batch
that creates and owns its lattices (lbm_create_batch, lbm_batch_member) and
the one-call adjoint (lbm_adjoint).  Each is checked bit for bit against the
calls it stands for, and the created batch and the one-call adjoint against
the FP64 oracle as well."""
import numpy as np
import pytest

from paper_2206_12412_gb300 import _abi as A
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


def _lattice_problem():
    p = W.base_problem(203, 61, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 50.0)
    return W.with_crack(p, mode="prescribed", y=30.0, x_tip=40.0, v_rel=0.4)


# ------------------------------------------------------------ strided copies

@pytest.mark.parametrize("storage", ["f64", "f32", "f32_lf", "f32_bf16", "f32_f16"])
@pytest.mark.parametrize("on_device", [False, True])
def test_strided_copies_match_the_dense_ones(gpu, storage, on_device):
    """Fields copied out with a row stride equal the dense copy in every row,
    the elements between rows stay untouched; fields set from a strided
    array give the same state (and the same next steps) as from the dense
    array."""
    import torch
    p = _lattice_problem()
    nx, ny, stride = p["nx"], p["ny"], p["nx"] + 13
    dt = np.float64 if storage == "f64" else np.float32
    code = A.STORAGE["f64"] if storage == "f64" else A.STORAGE["f32"]
    lat = gpu.Lattice(p, storage)
    w0, wd0 = W.random_state(nx, ny, seed=4, dtype=dt)
    lat.set_fields(w0, wd0)
    lat.step(37)
    dense = lat.fields()
    for k, which in enumerate(("w", "wdot")):
        if on_device:
            buf = torch.full((ny, stride), 7.0, dtype=torch.float64 if storage == "f64" else torch.float32, device="cuda")
            gpu.lbm_fields_strided(lat.h, A.FIELD[which], buf.data_ptr(), True, code, stride)
            torch.cuda.synchronize()
            got = buf.cpu().numpy()
        else:
            got = np.full((ny, stride), 7.0, dt)
            gpu.lbm_fields_strided(lat.h, A.FIELD[which], got.ctypes.data, False, code, stride)
        np.testing.assert_array_equal(got[:, :nx], dense[k])
        assert np.all(got[:, nx:] == 7.0)
    # set from strided arrays (junk between rows) and step on: the same bits
    # as a lattice set from the dense arrays
    ref = gpu.Lattice(p, storage)
    ref.set_fields(*dense)
    other = gpu.Lattice(p, storage)
    for k, which in enumerate(("w", "wdot")):
        src = np.full((ny, stride), np.nan, dt)
        src[:, :nx] = dense[k]
        if on_device:
            t = torch.from_numpy(src).cuda()
            gpu.lbm_set_fields_strided(other.h, A.FIELD[which], t.data_ptr(), True, code, stride)
            torch.cuda.synchronize()
        else:
            gpu.lbm_set_fields_strided(other.h, A.FIELD[which], src.ctypes.data, False, code, stride)
    for a, b in zip(other.fields(), ref.fields()):
        np.testing.assert_array_equal(a, b)
    ref.step(20)
    other.step(20)
    for a, b in zip(other.fields(), ref.fields()):
        np.testing.assert_array_equal(a, b)
    for L in (lat, ref, other):
        L.close()


def test_strided_copies_reject_a_short_stride(gpu):
    p = _lattice_problem()
    lat = gpu.Lattice(p, "f32")
    buf = np.zeros((p["ny"], p["nx"]), np.float32)
    with pytest.raises(gpu.LbmError) as ei:
        gpu.lbm_fields_strided(lat.h, A.FIELD["w"], buf.ctypes.data, False, A.STORAGE["f32"], p["nx"] - 1)
    assert ei.value.status == A.LBM_ERR_ARG
    with pytest.raises(gpu.LbmError):
        gpu.lbm_set_fields_strided(lat.h, A.FIELD["w"], buf.ctypes.data, False, A.STORAGE["f32"], 0)
    lat.close()


# ------------------------------------------------------- the created batch

def _batch_problems():
    return W.batch_problems(6, seed=11)


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_created_batch_matches_a_batch_of_handles(gpu, storage):
    """lbm_create_batch builds the same lattices as lbm_create and steps them
    as lbm_batch_create's batch does: every member bit-identical to the
    lattice of a batch made from separately created handles."""
    probs = [dict(p, hist_cap=512) for p in _batch_problems()]
    b = gpu.lbm_create_batch(probs, storage)
    lats = [gpu.Lattice(p, storage) for p in probs]
    ref = gpu.Batch(lats)
    gpu.lbm_batch_step(b, 150)
    ref.step(150)
    for i, (p, lat) in enumerate(zip(probs, lats)):
        view = gpu.SlabView(gpu.lbm_batch_member(b, i), p, storage, 0, p["ny"])
        for x, y in zip(view.fields(), lat.fields()):
            np.testing.assert_array_equal(x, y)
        assert view.crack_state() == lat.crack_state()
        np.testing.assert_array_equal(view.cut_mask("v"), lat.cut_mask("v"))
    with pytest.raises(gpu.LbmError):
        gpu.lbm_batch_member(b, len(probs))
    gpu.lbm_batch_destroy(b)   # destroys its own lattices too
    ref.close()
    for lat in lats:
        lat.close()


def test_created_batch_matches_the_oracle(oracle_mod, gpu):
    """FP64 members of a created batch against the oracle's runs of the same
    problems: fields within 1e-12 relative max-norm, tips and severed links
    exact (prescribed growth)."""
    probs = [dict(p, hist_cap=512) for p in _batch_problems() if p["crack"]["mode"] == "prescribed"][:3]
    probs = [dict(p, nx=min(p["nx"], 320), ny=min(p["ny"], 160)) for p in probs]
    probs = [dict(p, crack=dict(p["crack"], y=float(p["ny"] // 2), x_tip=min(p["crack"]["x_tip"], 0.3 * p["nx"])))
             for p in probs]
    b = gpu.lbm_create_batch(probs, "f64")
    gpu.lbm_batch_step(b, 120)
    for i, p in enumerate(probs):
        o = oracle_mod.Oracle(p)
        o.step(120)
        view = gpu.SlabView(gpu.lbm_batch_member(b, i), p, "f64", 0, p["ny"])
        wo, wdo = o.fields()
        wg, wdg = view.fields()
        scale = max(np.abs(wo).max(), 1e-300)
        assert np.abs(wg - wo).max() <= 1e-12 * scale and np.abs(wdg - wdo).max() <= 1e-12 * scale
        assert view.crack_state()["tip_q"] == o.crack()["tip_q"]
        np.testing.assert_array_equal(view.cut_mask("v"), o.cuts()[1].astype(bool))
        o.close()
    gpu.lbm_batch_destroy(b)


def test_created_batch_names_the_member_that_fails(gpu):
    probs = _batch_problems()[:3]
    bad = dict(probs[1], mu=-1.0)
    with pytest.raises(gpu.LbmError) as ei:
        gpu.lbm_create_batch([probs[0], bad, probs[2]], "f32")
    assert ei.value.status == A.LBM_ERR_ARG and "lattice 1" in str(ei.value)


# ------------------------------------------------------- the one-call adjoint

@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("every", [0, 10])
def test_one_call_adjoint_matches_the_tape(gpu, storage, every):
    """lbm_adjoint returns the loss and gradients of the tape sequence it
    stands for, bit for bit, stored or checkpointed."""
    T = 60
    p, _, w0, wd0, sens, tgt = W.adjoint_case("macro_growth", T, seed=21, ns=6)
    a = gpu.Lattice(p, storage)
    a.set_fields(w0, wd0)
    tape = gpu.Tape(a, sens, T, checkpoint_every=every)
    loss_t = tape.forward(tgt)
    dl_t, dw_t, dwd_t = tape.backward(device=False)
    tape.close()
    bl = gpu.Lattice(p, storage)
    bl.set_fields(w0, wd0)
    loss_c, dl_c, dw_c, dwd_c = gpu.lbm_adjoint(bl, sens, T, tgt, checkpoint_every=every)
    assert loss_c == loss_t
    np.testing.assert_array_equal(dl_c, dl_t)
    np.testing.assert_array_equal(dw_c, dw_t)
    np.testing.assert_array_equal(dwd_c, dwd_t)
    # the handle ends T steps on, as after the tape's forward run
    for x, y in zip(bl.fields(), a.fields()):
        np.testing.assert_array_equal(x, y)
    a.close()
    bl.close()


def test_one_call_adjoint_matches_the_oracle(oracle_mod, gpu):
    T = 80
    p, _, w0, wd0, sens, tgt = W.adjoint_case("bb_growth", T, seed=21, ns=6)
    ref = oracle_mod.adjoint(p, T, sens, tgt, w0, wd0)
    lat = gpu.Lattice(p, "f64")
    lat.set_fields(w0, wd0)
    loss, dload, dw, dwd = gpu.lbm_adjoint(lat, sens, T, tgt)
    assert loss == pytest.approx(ref["loss"], rel=1e-12)
    for got, key in ((dload, "dload"), (dw, "dw0"), (dwd, "dwd0")):
        r = np.asarray(ref[key])
        assert np.abs(got - r).max() <= 1e-10 * max(np.abs(r).max(), 1e-300), key
    lat.close()
