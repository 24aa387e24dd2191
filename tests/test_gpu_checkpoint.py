"""Checkpoint / resume (include/lbm.h: lbm_save, lbm_load): a run saved at
step n and resumed in a fresh handle gives the same bits as the run that
went on -- fields, cut masks, both crack ends, the history ring -- for each
storage form and for a K-criterion two-tip crack under the macroscopic rule
on every boundary; and the calls fail cleanly on a wrong configuration, a
missing file, a truncated file and a file that is no checkpoint."""
import os

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


def _problem(kind):
    if kind == "centre":
        return W.kcrit_centre_crack(scale=2)
    p = W.base_problem(300, 80, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=40.0, x_tip=50.0, v_rel=0.5)
    return W.with_antisymmetric_ramp(p, 1e-3, 60.0)


def _same(a, b):
    wa, wda = a.fields()
    wb, wdb = b.fields()
    np.testing.assert_array_equal(wb, wa)
    np.testing.assert_array_equal(wdb, wda)
    np.testing.assert_array_equal(b.cut_mask("v"), a.cut_mask("v"))
    assert b.crack_state() == a.crack_state()
    ha, hb = a.history(), b.history()
    for k in ha:
        np.testing.assert_array_equal(hb[k], ha[k])


@pytest.mark.parametrize("kind,storage", [("centre", "f32"), ("centre", "f64"), ("strip", "f32_f16"),
                                          ("strip", "f32_bf16")])
def test_resume_gives_the_same_bits(gpu, tmp_path, kind, storage):
    p = _problem(kind)
    path = str(tmp_path / "state.lbm")
    a = gpu.Lattice(p, storage)
    a.step(300)                     # graph chunks and single launches
    a.save(path)
    a.step(701)
    b = gpu.Lattice(p, storage)
    b.step(5)                       # a state of its own, replaced by the load
    b.load(path)
    b.step(701)
    _same(a, b)
    if p["crack"].get("two_tips"):
        assert b.crack_state_left() == a.crack_state_left()
    a.close()
    b.close()


def test_load_rejects_bad_files_and_configurations(gpu, tmp_path):
    p = _problem("strip")
    a = gpu.Lattice(p, "f32")
    a.step(10)
    path = str(tmp_path / "s.lbm")
    a.save(path)
    other = gpu.Lattice(dict(p, nx=301), "f32")
    with pytest.raises(gpu.LbmError) as ei:
        other.load(path)
    assert ei.value.status == gpu.A.LBM_ERR_ARG
    f64 = gpu.Lattice(p, "f64")
    with pytest.raises(gpu.LbmError):
        f64.load(path)
    with pytest.raises(gpu.LbmError) as ei:
        a.load(str(tmp_path / "missing.lbm"))
    assert ei.value.status == gpu.A.LBM_ERR_IO
    with open(path, "rb") as f:
        data = f.read()
    cut = str(tmp_path / "cut.lbm")
    with open(cut, "wb") as f:
        f.write(data[: len(data) // 2])
    with pytest.raises(gpu.LbmError) as ei:
        a.load(cut)
    assert ei.value.status == gpu.A.LBM_ERR_IO
    junk = str(tmp_path / "junk.lbm")
    with open(junk, "wb") as f:
        f.write(os.urandom(4096))
    with pytest.raises(gpu.LbmError) as ei:
        a.load(junk)
    assert ei.value.status == gpu.A.LBM_ERR_IO
    with pytest.raises(gpu.LbmError) as ei:
        a.save(str(tmp_path / "no_such_dir" / "s.lbm"))
    assert ei.value.status == gpu.A.LBM_ERR_IO
    # the handle is still usable after the failed calls
    a.step(5)
    for l in (a, other, f64):
        l.close()
