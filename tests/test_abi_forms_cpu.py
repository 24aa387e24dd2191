"""Argument checks of the C-ABI call forms that take the state in other
shapes (strided field copies, the batch that creates its lattices, the
one-call adjoint): every rejection here happens before any CUDA call, so it
runs without a GPU."""
import ctypes as C

import pytest

from paper_2206_12412_gb300 import _abi as A
from paper_2206_12412_gb300 import lbm
from paper_2206_12412_gb300 import workloads as W


@pytest.fixture(scope="module")
def lib():
    return lbm.load_library()


def _status(rc: int) -> str:
    return A.STATUS_NAMES.get(rc, str(rc))


def test_strided_copies_reject_a_null_handle(lib):
    buf = (C.c_float * 16)()
    assert lib.lbm_fields_strided(None, 0, buf, 0, A.STORAGE["f32"], 8) == A.LBM_ERR_ARG
    assert lib.lbm_set_fields_strided(None, 0, buf, 0, A.STORAGE["f32"], 8) == A.LBM_ERR_ARG
    assert "NULL" in lib.lbm_last_error().decode()


def test_created_batch_rejects_bad_arrays(lib):
    out = C.c_void_p()
    g, lat, mat = A.Grid(), A.Lattice_(), A.Material()
    assert lib.lbm_create_batch(0, C.byref(g), C.byref(lat), C.byref(mat), None, None, None, None, None, 0,
                                C.byref(out)) == A.LBM_ERR_ARG
    assert "n >= 1" in lib.lbm_last_error().decode()
    n_loads = (C.c_int32 * 1)(0)
    assert lib.lbm_create_batch(1, C.byref(g), C.byref(lat), C.byref(mat), None, None, n_loads, None, None, 0,
                                C.byref(out)) == A.LBM_ERR_ARG
    assert "together" in lib.lbm_last_error().decode()
    assert out.value is None


def test_created_batch_names_the_member_that_fails(lib):
    """Member 0 fails lbm_create's argument checks (before any device call):
    the batch reports it by index and leaves nothing behind."""
    bad = dict(W.base_problem(64, 32), mu=-1.0)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_batch([bad, W.base_problem(64, 32)], "f32")
    assert ei.value.status == A.LBM_ERR_ARG, _status(ei.value.status)
    assert "lattice 0" in str(ei.value) and "mu" in str(ei.value)


def test_batch_member_rejects_null(lib):
    h = C.c_void_p()
    assert lib.lbm_batch_member(None, 0, C.byref(h)) == A.LBM_ERR_ARG


def test_one_call_adjoint_rejects_a_null_handle(lib):
    sens = (C.c_int32 * 2)(1, 1)
    tg = (C.c_double * 4)()
    loss = C.c_double()
    rc = lib.lbm_adjoint(None, sens, 1, 4, 0, tg, 0, C.byref(loss), None, 0, None, None, 0, A.STORAGE["f32"], None)
    assert rc == A.LBM_ERR_ARG, _status(rc)
