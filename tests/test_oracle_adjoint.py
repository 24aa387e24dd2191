"""Pins of the oracle's adjoint (the transposed steps) to things other than
itself: central differences of the oracle's forward run (the misfit is
quadratic in the loads and initial fields once the cut schedule is fixed, so
central differences are exact up to rounding), a full brute-force gradient on
a tiny lattice, and closed forms of one step.  The forward run is pinned by
test_oracle_pins.py."""
import numpy as np
import pytest

import oracle
from paper_2206_12412_gb300 import workloads as W


def _case(kind: str, T: int, seed: int):
    return W.adjoint_case(kind, T, seed)


def _loss(p, T, sens, tgt, w0, wd0):
    return oracle.adjoint(p, T, sens, tgt, w0, wd0, grad=False)["loss"]


def _series(p, e):
    return next(ld["series"] for ld in p["loads"] if ld["edge"] == e)


@pytest.mark.parametrize("kind", ["macro_growth", "bb_growth", "bb_periodic", "all_dirichlet", "scaled_units", "no_crack"])
def test_adjoint_matches_central_differences(kind):
    """<grad L, d> equals (L(x + eps d) - L(x - eps d)) / (2 eps) of the
    forward run along random directions of the loads and initial fields."""
    T = 40
    p, loaded, w0, wd0, sens, tgt = _case(kind, T, seed=11)
    r = oracle.adjoint(p, T, sens, tgt, w0, wd0)
    rng = np.random.default_rng(5)
    for trial in range(3):
        d_w = 1e-3 * rng.standard_normal(w0.shape)
        d_wd = 1e-4 * rng.standard_normal(w0.shape)
        d_u = {e: 1e-3 * rng.standard_normal(T) for e in loaded}
        pred = float(np.sum(r["dw0"] * d_w) + np.sum(r["dwd0"] * d_wd))
        for e, d in d_u.items():
            pred += float(np.dot(r["dload"][oracle.EDGE_INDEX[e]], d))
        Ls = []
        for sgn in (1.0, -1.0):
            q = p
            for e, d in d_u.items():
                q = W.with_series_load(q, e, _series(p, e) + sgn * d)
            Ls.append(_loss(q, T, sens, tgt, w0 + sgn * d_w, wd0 + sgn * d_wd))
        fd = (Ls[0] - Ls[1]) / 2.0
        assert fd == pytest.approx(pred, rel=1e-9, abs=1e-9 * abs(r["loss"])), (kind, trial)
    # edges without a Dirichlet condition get no load gradient
    for e, ix in oracle.EDGE_INDEX.items():
        if p["edges"][ix] != "dirichlet":
            assert not np.any(r["dload"][ix])


def test_adjoint_brute_force_gradient_tiny():
    """Every component of dL/dw0 and dL/dwdot0 on a 9 x 8 lattice with a
    growing macroscopic crack, by central differences one site at a time."""
    T = 7
    p = W.base_problem(9, 8, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=4.0, x_tip=2.0, v_rel=0.8)
    rng = np.random.default_rng(3)
    p = W.with_series_load(p, "top", 1e-3 * rng.standard_normal(T))
    w0 = 1e-3 * rng.standard_normal((8, 9))
    wd0 = 1e-4 * rng.standard_normal((8, 9))
    sens = np.array([[1, 3], [4, 4], [6, 1], [2, 6]], np.int32)
    tgt = 1e-3 * rng.standard_normal((T, 4))
    r = oracle.adjoint(p, T, sens, tgt, w0, wd0)
    eps = 1e-3
    g_w = np.zeros_like(w0)
    g_wd = np.zeros_like(w0)
    for j in range(8):
        for i in range(9):
            e = np.zeros_like(w0)
            e[j, i] = eps
            g_w[j, i] = (_loss(p, T, sens, tgt, w0 + e, wd0) - _loss(p, T, sens, tgt, w0 - e, wd0)) / (2 * eps)
            g_wd[j, i] = (_loss(p, T, sens, tgt, w0, wd0 + e) - _loss(p, T, sens, tgt, w0, wd0 - e)) / (2 * eps)
    scale = max(np.abs(g_w).max(), 1e-300)
    assert np.abs(r["dw0"] - g_w).max() <= 1e-8 * scale
    assert np.abs(r["dwd0"] - g_wd).max() <= 1e-8 * max(np.abs(g_wd).max(), 1e-300)
    # and for each load value of the top edge
    u = _series(p, "top")
    for n in range(T):
        e = np.zeros(T)
        e[n] = eps
        Lp = _loss(W.with_series_load(p, "top", u + e), T, sens, tgt, w0, wd0)
        Lm = _loss(W.with_series_load(p, "top", u - e), T, sens, tgt, w0, wd0)
        assert r["dload"][3, n] == pytest.approx((Lp - Lm) / (2 * eps), rel=1e-8, abs=1e-12 * scale)


def test_adjoint_one_step_closed_form():
    """One step without a crack: w^1_s = w_s + dt (wdot_s + g (sum_nb w - 4 w_s)),
    so dL/dw0 is 2 r (1 - 4 g dt) at the sensor and 2 r g dt at each
    neighbour, dL/dwdot0 = 2 r dt, with r the misfit of w^1_s.  A sensor next
    to the top Dirichlet edge (anti-bounce-back value 2 w* - w_s) also has
    dL/dw*_top(t_0) = 2 r (2 g dt) and a diagonal 2 r (1 - 5 g dt)."""
    p = W.base_problem(10, 9, edges=("free", "free", "dirichlet", "dirichlet"))
    p = W.with_series_load(p, "top", np.array([2e-3]))
    rng = np.random.default_rng(8)
    w0 = 1e-3 * rng.standard_normal((9, 10))
    wd0 = 1e-4 * rng.standard_normal((9, 10))
    g, dt = 0.25, 1.0
    for (i, j), top in (((4, 4), False), ((6, 8), True)):
        sens = np.array([[i, j]], np.int32)
        tgt = np.array([[3e-4]])
        r = oracle.adjoint(p, 1, sens, tgt, w0, wd0)
        res = r["trace"][0, 0] - tgt[0, 0]
        diag = 1 - (5 if top else 4) * g * dt
        exp_w = np.zeros((9, 10))
        exp_w[j, i] = 2 * res * diag
        for di, dj in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            if 0 <= j + dj < 9:
                exp_w[j + dj, i + di] = 2 * res * g * dt
        np.testing.assert_allclose(r["dw0"], exp_w, rtol=1e-12, atol=1e-20)
        exp_wd = np.zeros((9, 10))
        exp_wd[j, i] = 2 * res * dt
        np.testing.assert_allclose(r["dwd0"], exp_wd, rtol=1e-12, atol=1e-20)
        assert r["dload"][3, 0] == pytest.approx(2 * res * 2 * g * dt if top else 0.0, rel=1e-12, abs=1e-20)
        assert r["loss"] == pytest.approx(res * res, rel=1e-12)


def test_adjoint_loss_and_trace_follow_the_forward_run():
    """The loss and trace reported with the gradient are those of a plain
    oracle run of the same problem."""
    T = 25
    p, _, w0, wd0, sens, tgt = _case("macro_growth", T, seed=2)
    r = oracle.adjoint(p, T, sens, tgt, w0, wd0)
    o = oracle.Oracle(p)
    o.set_fields(w0, wd0)
    tr = np.zeros((T, len(sens)))
    for n in range(T):
        o.step(1)
        w, _ = o.fields()
        tr[n] = w[sens[:, 1], sens[:, 0]]
    np.testing.assert_array_equal(r["trace"], tr)
    assert r["loss"] == pytest.approx(float(np.sum((tr - tgt) ** 2)), rel=1e-14)
