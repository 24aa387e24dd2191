"""Pins of the oracle's two-tip crack (both ends of a centre crack grow, as
in the paper's K-criterion example, Sec. 5.2): exact prescribed growth of
both ends with the closed-segment cuts of Alg. 1, K at a left end from a
synthetic near-tip field, and the mirror symmetry of a centred crack."""
import math

import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W


def _cuts(nx, ny, jc, x_lo, x_hi):
    """Severed V links of a straight crack on y = jc from x_lo to x_hi
    (closed segment: x_i = i + 1/2 in [x_lo, x_hi])."""
    cv = np.zeros((ny, nx), bool)
    for i in range(nx):
        if x_lo <= i + 0.5 <= x_hi:
            cv[jc - 1, i] = True
    return cv


@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_prescribed_two_tips_advance_and_cut(oracle_mod, bc_mode):
    """Both ends move by the nearest 2^-32 dh step to Delta a = v c_s dt per
    step, the left one towards -x, each stopping at its far edge; the severed
    links are exactly those between the two ends."""
    nx, ny, jc = 60, 16, 8
    p = W.base_problem(nx, ny, bc_mode=bc_mode)
    p = W.with_crack(p, mode="prescribed", y=float(jc), x_start=25.3, x_tip=33.1, v_rel=0.55, two_tips=True)
    p = W.with_antisymmetric_ramp(p, 1e-3, 10.0)
    o = oracle_mod.Oracle(p)
    dq = round(0.55 * 0.5 * 2**32)
    r0, l0 = round(33.1 * 2**32), round(25.3 * 2**32)
    for n in range(1, 131):
        o.step(1)
        right = min(r0 + n * dq, nx * 2**32)
        left = max(l0 - n * dq, 0)
        assert o.crack()["tip_q"] == right
        assert o.left_tip_q() == left
        _, cv = o.cuts()
        assert np.array_equal(cv.astype(bool), _cuts(nx, ny, jc, left / 2**32, right / 2**32)), n
    assert o.crack()["flags"] & 1   # stopped at the edges
    h, hl = o.history(), o.history_left()
    assert np.all(hl["tip_q"] == np.maximum(l0 - np.arange(1, 131) * dq, 0))
    assert hl["grew"].sum() == math.ceil(l0 / dq) and h["grew"].sum() == math.ceil((nx * 2**32 - r0) / dq)
    # the boundary points are the sites next to every severed link
    cols = np.nonzero(cv[jc - 1])[0]
    assert set(o.bpoints().tolist()) == {jc * nx + i for i in cols} | {(jc - 1) * nx + i for i in cols}


@pytest.mark.parametrize("r_min,fit", [(2.0, 1.0), (1.5, 3.0)])
def test_K_at_a_left_tip_from_a_near_tip_field(oracle_mod, r_min, fit):
    """The mode III near-tip field of an end pointing towards -x, written as
    the mirror image of the right-end field (same opening w(above) -
    w(below) = (4K/mu) sqrt(r/2pi) at distance r behind the tip), returns K."""
    nx, ny, jc = 60, 20, 10
    p = W.base_problem(nx, ny)
    p = W.with_crack(p, mode="stationary", y=float(jc), x_start=17.63, x_tip=50.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    mu, K = p["mu"], 0.29
    ltip = o.left_tip_q()
    w = np.zeros((ny, nx))
    for i in range(nx):
        r = (i + 0.5) - ltip / 2**32
        if r <= 0:
            continue
        amp = 2 * K / mu * math.sqrt(r / (2 * math.pi))
        w[jc, i], w[jc - 1, i] = amp, -amp
    Kc, npairs = o.evaluate_K_left(w, ltip, r_min, fit)
    assert npairs == sum(1 for i in range(nx) if r_min <= (i + 0.5) - ltip / 2**32 < r_min + fit)
    assert abs(Kc - K) < 1e-13 * K
    # the right-end evaluation of the same field sees nothing of the left end
    Kr, npr = o.evaluate_K(w, o.crack()["tip_q"], r_min, fit)
    assert npr >= 1 and abs(Kr - K) > 0.1 * K


@pytest.mark.parametrize("bc_mode", ["macroscopic", "bounceback"])
def test_centred_crack_grows_mirror_symmetrically(oracle_mod, bc_mode):
    """A crack centred in a lattice whose edges and loads are mirror
    symmetric in x: under the K-criterion both ends see the same K (to
    rounding), start growing in the same step and stay mirror images."""
    nx, ny = 96, 48
    p = W.base_problem(nx, ny, bc_mode=bc_mode)
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_start=38.0, x_tip=58.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    o.step(400)
    h, hl = o.history(), o.history_left()
    assert h["grew"].sum() > 10 and hl["grew"].sum() == h["grew"].sum()
    np.testing.assert_array_equal(hl["grew"], h["grew"])
    np.testing.assert_allclose(hl["K"], h["K"], rtol=1e-9, atol=1e-12 * np.abs(h["K"]).max())
    # mirror images on the 2^-32 grid, to a few units of it
    assert np.abs((nx * 2**32 - hl["tip_q"]) - h["tip_q"]).max() <= 16
    _, cv = o.cuts()
    np.testing.assert_array_equal(cv, cv[:, ::-1])


def test_each_tip_uses_its_own_previous_speed(oracle_mod):
    """An off-centre crack: the ends grow at different speeds.  At every step
    the left end's K is eq. sif over the pairs behind it at r_min = r0 / (1 -
    v_prev) with ITS OWN previous speed (eq. r(v)), evaluated on the fields
    after the LBM step."""
    nx, ny = 120, 48
    p = W.base_problem(nx, ny, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.45 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_start=30.0, x_tip=70.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    ltip_prev, vl_prev, checked = o.left_tip_q(), 0.0, 0
    for n in range(300):
        o.step(1)
        w, _ = o.fields()
        hl = o.history_left()
        K_exp, np_exp = o.evaluate_K_left(w, ltip_prev, 2.0 / (1.0 - vl_prev), 1.0)
        assert hl["npairs"][n] == np_exp
        assert hl["K"][n] == pytest.approx(K_exp, rel=1e-14, abs=1e-300)
        checked += vl_prev > 0
        ltip_prev, vl_prev = hl["tip_q"][n], hl["v"][n]
    h = o.history()
    assert checked > 5 and not np.array_equal(h["v"], hl["v"])   # both grew, at different speeds
