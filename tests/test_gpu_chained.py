"""Chained launches (include/lbm.h: lbm_set_chained, lbm_batch_set_chained;
programmatic dependent launch between the kernels of consecutive steps)
change only when a kernel starts, never what it computes: every path steps
to the same bits chained and plain -- D2Q5 with the edge rule, leapfrog
storage, D2Q9 with its crack-face kernel, a crack in another direction with
its face solve, a batch with edge-rule units -- through graph chunks and
single launches, and the chained run still meets the oracle."""
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
    assert np.array_equal(wa, wb) and np.array_equal(wda, wdb)
    assert a.crack_state() == b.crack_state()


def _d2q9():
    p = W.base_problem(300, 40, bc_mode="macroscopic")
    p["lattice"] = "D2Q9"
    p = W.with_crack(p, mode="prescribed", y=20.0, x_start=120.3, x_tip=160.6, v_rel=0.6, two_tips=True)
    return W.with_antisymmetric_ramp(p, 1e-3, 50.0)


CASES = {
    "sec52_edge_rule_f32": (lambda: W.kcrit_centre_crack(scale=2), "f32"),
    "sec52_edge_rule_f64": (lambda: W.kcrit_centre_crack(scale=2), "f64"),
    "kcrit_leapfrog": (lambda: W.kcrit_single(scale=16), "f32_lf"),
    "kcrit_bf16": (lambda: W.kcrit_single(scale=16), "f32_bf16"),
    "d2q9_faces": (_d2q9, "f32"),
    "line_macro_faces": (lambda: W.kcrit_line_centre(scale=8), "f32"),
    "line_link_local": (lambda: W.kcrit_line(scale=8), "f32"),
}


@pytest.mark.parametrize("case", sorted(CASES))
def test_chained_and_plain_launches_give_the_same_bits(gpu, case):
    make, storage = CASES[case]
    p = make()
    chained = gpu.Lattice(p, storage)
    plain = gpu.Lattice(p, storage)
    chained.set_chained(True)
    plain.set_chained(False)
    for n in (3, 64, 130, 1):
        chained.step(n)
        plain.step(n)
    _same(chained, plain)
    chained.close()
    plain.close()


def test_chained_batch_gives_the_solo_bits(gpu):
    ps = W.batch_problems(6, seed=5) + [W.kcrit_centre_crack(scale=2)]
    solo = [gpu.Lattice(p, "f32") for p in ps]
    mem = [gpu.Lattice(p, "f32") for p in ps]
    for s in solo:
        s.set_chained(False)
    b = gpu.Batch(mem)
    b.set_chained(True)
    b.step(3)
    b.step(128)
    b.set_chained(False)
    b.step(5)
    for s in solo:
        s.step(136)
    for s, m in zip(solo, mem):
        _same(s, m)
    b.close()


def test_chained_run_meets_the_oracle(oracle_mod, gpu):
    p = W.kcrit_centre_crack(scale=4)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f64")
    g.set_chained(True)
    for n in (7, 64, 129):
        o.step(n)
        g.step(n)
    wo, wdo = o.fields()
    wg, wdg = g.fields()
    scale = max(np.abs(wo).max(), 1e-300)
    assert np.abs(wg - wo).max() <= 1e-12 * scale
    assert np.abs(wdg - wdo).max() <= 1e-12 * scale
    np.testing.assert_array_equal(g.history()["tip_q"], o.history()["tip_q"])
    np.testing.assert_array_equal(g.history_left()["tip_q"], o.history_left()["tip_q"])
    g.close()
    o.close()
