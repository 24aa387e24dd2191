"""The record CTA of the step kernel: a CTA of its own that runs the crack
step of Alg. 1 beside the rows when the rows next to the crack do not need
its decision.  With a prescribed speed the decision needs no K, so the crack
sub-band CTAs advance the tip at once and the record CTA forms the K of the
history (eq. sif).  With the K-criterion, a step whose tip cannot reach the
next link to sever even at v_max leaves those rows unchanged whatever K is,
so the record CTA runs the whole step (K fit, eq. v-tanh, advance) while the
rows are updated; otherwise the sub-band CTAs run it first, as before.  The
batched kernel always runs the whole step in the sub-band CTA, so a batch of
one lattice is the reference: every field, mask, state and history entry --
K, pair counts and r_min included -- must be bit-identical, also when host
reads apply the deferred crack step between launches, for one and two
growing ends, FP64 and FP32, and in the adjoint's recording steps."""
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


def _problems():
    a = W.adjoint_problem(nx=1024, ny=1024, n_steps=400, ns=8)["problem"]
    b = W.base_problem(300, 96, bc_mode="bounceback")
    b = W.with_antisymmetric_ramp(b, 2e-3, 100.0)
    b = W.with_crack(b, mode="prescribed", y=48.0, x_start=120.0, x_tip=160.0, v_rel=0.6, two_tips=True, r0=3.0)
    c = W.base_problem(128, 128, bc_mode="macroscopic")
    c = W.with_antisymmetric_ramp(c, 1e-3, 200.0)
    c = W.with_crack(c, mode="prescribed", y=64.0, x_tip=32.0, v_rel=0.3)
    return {"adjoint_1024": a, "two_tips": b, "c1_128": c}


def _same(a, b, two_tips=False):
    for x, y in zip(a.fields(), b.fields()):
        np.testing.assert_array_equal(x, y)
    np.testing.assert_array_equal(a.cut_mask("v"), b.cut_mask("v"))
    assert a.crack_state() == b.crack_state()
    for ha, hb in ((a.history(), b.history()),) + (((a.history_left(), b.history_left()),) if two_tips else ()):
        for k in ha:
            np.testing.assert_array_equal(ha[k], hb[k], err_msg=k)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["adjoint_1024", "two_tips", "c1_128"])
def test_record_cta_gives_the_bits_of_the_whole_crack_step(gpu, storage, kind):
    p = _problems()[kind]
    solo = gpu.Lattice(p, storage)
    ref_lat = gpu.Lattice(p, storage)
    ref = gpu.Batch([ref_lat])
    solo.step(1)
    ref.step(1)
    solo.step(130)    # graph chunks
    ref.step(130)
    h = solo.history()
    assert (h["v"] > 0).all() and (h["npairs"] > 0).any()
    # host reads between single steps: each read applies the pending crack
    # step, so the next launch finds it decided and carries its K over
    for _ in range(5):
        solo.step(1)
        solo.crack_state()
        ref.step(1)
    solo.step(70)
    ref.step(70)
    _same(solo, ref_lat, two_tips=p["crack"].get("two_tips", False))
    ref.close()
    solo.close()
    ref_lat.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["macro_growth", "wide_bb"])
def test_record_cta_in_the_adjoint_recording(gpu, storage, kind):
    """The tape's recording steps take the record CTA too: the recorded
    lattice ends with the fields, state and history (K included) of a batch
    of one stepped from the same state with the same loads."""
    T = 120
    p, _, w0, wd0, sens, tgt = W.adjoint_case(kind, T, seed=5, ns=6)
    lat = gpu.Lattice(p, storage)
    lat.set_fields(w0, wd0)
    tape = gpu.Tape(lat, sens, T)
    tape.forward(tgt)
    ref_lat = gpu.Lattice(p, storage)
    ref_lat.set_fields(w0, wd0)
    ref = gpu.Batch([ref_lat])
    ref.step(T)
    _same(lat, ref_lat)
    tape.close()
    ref.close()
    lat.close()
    ref_lat.close()


def _kcrit_problems():
    a = W.kcrit_single(scale=8)                 # 512 x 256, one end, macroscopic faces
    b = W.kcrit_centre_crack(scale=2)           # Sec. 5.2 at half size: two ends, the rule on every boundary
    c = W.kcrit_single(scale=8, bc_mode="bounceback")
    return {"kcrit_single": (a, 900), "sec52_half": (b, W.KCRIT_CENTRE_STEPS // 2), "kcrit_bb": (c, 900)}


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind", ["kcrit_single", "sec52_half", "kcrit_bb"])
def test_kcrit_steps_out_of_reach_give_the_bits_of_the_whole_crack_step(gpu, storage, kind):
    p, n = _kcrit_problems()[kind]
    p = dict(p, hist_cap=max(n + 16, 4096))
    solo = gpu.Lattice(p, storage)
    ref_lat = gpu.Lattice(p, storage)
    ref = gpu.Batch([ref_lat])
    solo.step(1)
    ref.step(1)
    solo.step(n - 40)
    ref.step(n - 40)
    for _ in range(5):       # host reads between single steps
        solo.step(1)
        solo.crack_state()
        ref.step(1)
    solo.step(34)
    ref.step(34)
    two = p["crack"].get("two_tips", False)
    h = solo.history(cap=n)
    assert (h["v"] > 0).sum() > 3, "the crack should grow in this run"
    _same(solo, ref_lat, two_tips=two)
    ref.close()
    solo.close()
    ref_lat.close()
