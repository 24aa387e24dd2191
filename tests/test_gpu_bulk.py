"""The bulk-copy march of the step kernel (lbm_set_bulk): interior CTAs that
stage their rows in shared memory by cp.async.bulk copies on mbarriers give
the same bits as the register march -- fields, masks, crack state and
history -- on lattices with many interior column blocks and bands, in every
FP32-w storage form, with both crack-face modes; and the oracle's run within
the parity tolerance."""
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


def _same(a, b):
    wa, wda = a.fields()
    wb, wdb = b.fields()
    np.testing.assert_array_equal(wa, wb)
    np.testing.assert_array_equal(wda, wdb)
    np.testing.assert_array_equal(a.cut_mask("v"), b.cut_mask("v"))
    assert a.crack_state() == b.crack_state()
    ha, hb = a.history(), b.history()
    for k in ha:
        np.testing.assert_array_equal(ha[k], hb[k])


def _pair(gpu, p, storage, seed):
    a = gpu.Lattice(p, storage)
    b = gpu.Lattice(p, storage)
    b.set_bulk(True)
    if storage == "f32_f16":
        # the loads' scale (2^32 here) is for their slow ramp: the random
        # state's wdot (about 1e-3) needs a smaller one to stay finite in FP16
        a.set_wd_scale(1024.0)
        b.set_wd_scale(1024.0)
    init = W.random_state(p["nx"], p["ny"], seed=seed, dtype=np.float32)
    a.set_fields(*init)
    b.set_fields(*init)
    return a, b


@pytest.mark.parametrize("storage", ["f32", "f32_bf16", "f32_f16"])
def test_bulk_march_full_size_benchmark_lattice(gpu, storage):
    p = W.kcrit_single()
    a, b = _pair(gpu, p, storage, 31)
    for n in (1, 11, 64):   # single launches and a graph chunk
        a.step(n)
        b.step(n)
    _same(a, b)
    a.close()
    b.close()


@pytest.mark.parametrize("bc", ["macroscopic", "bounceback"])
@pytest.mark.parametrize("band_rows", [0, 7, 40])
def test_bulk_march_prescribed_growth_any_band_height(gpu, bc, band_rows):
    p = W.base_problem(2100, 230, bc_mode=bc, edges=("dirichlet", "free", "dirichlet", "dirichlet"))
    p = W.with_antisymmetric_ramp(p, 2e-3, 50.0)
    p = W.with_crack(p, mode="prescribed", y=115.0, x_tip=300.0, v_rel=0.6)
    a, b = _pair(gpu, p, "f32", 5)
    if band_rows:
        a.set_launch(band_rows)
        b.set_launch(band_rows)
    a.step(150)
    b.step(150)
    _same(a, b)
    a.close()
    b.close()


def test_bulk_march_matches_the_oracle(oracle_mod, gpu):
    from test_gpu_parity import compare_crack, compare_fields, compare_masks
    p = W.base_problem(1100, 130, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 130.0)
    p = W.with_crack(p, mode="kcrit", y=65.0, x_tip=200.0, K_C=K_C, v_max=0.85, r0=2.0)
    g = gpu.Lattice(p, "f32")
    g.set_bulk(True)
    o = oracle_mod.Oracle(p)
    init = W.random_state(p["nx"], p["ny"], seed=3, dtype=np.float32)
    g.set_fields(*init)
    o.set_fields(*init)
    g.step(200)
    o.step(200)
    compare_fields(o, g, "f32")
    ho, hg = o.history(), g.history()
    assert np.abs(hg["tip_q"] - ho["tip_q"]).max() < 2**32
    o.close()
    g.close()
