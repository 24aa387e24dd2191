"""Pins of the oracle's D2Q9 lattice (the paper notes that the crack
handling carries over to D2Q9; Sec. 4.1), with link-local boundaries and
with the macroscopic rule on the crack faces.

Equilibrium read as f_eq^a = W_a g w with W = 2/3 along the axes and 1/6
along the diagonals (the isotropic nine-point Laplacian; axis weight plus
twice the diagonal weight is 1, so the wave speed is c_s), f_eq^0 = wdot
minus their sum.  With tau = dt the scheme is the leapfrog
    w^{n+1} - 2 w^n + w^{n-1} = g L9 w^n,
whose Fourier symbol gives the closed-form discrete dispersion relation
    cos(Omega dt) = 1 - S(k) / 2,
    S(k) = g [2/3 (4 - 2 cos kx - 2 cos ky) + 1/6 (4 - 2 cos(kx + ky) - 2 cos(kx - ky))],
stable while max S = 16 g / 3 <= 4, i.e. g dt <= 3/4.  Links: the diagonal
links between rows jc-1 and jc cross the crack line at x = i + 1 and are
severed when that point lies on the closed crack segment; a missing link
takes bounce-back (free edge, crack) or anti-bounce-back with its own weight
(Dirichlet), a diagonal through a corner of the body the Dirichlet edge's
rule if just one of the two is Dirichlet, else the bottom / top edge's."""
import math

import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

WA, WD = 2.0 / 3.0, 1.0 / 6.0


def _problem(nx, ny, edges=("free", "free", "dirichlet", "dirichlet"), cs=0.5):
    p = W.base_problem(nx, ny, bc_mode="bounceback", edges=edges, cs=cs)
    p["lattice"] = "D2Q9"
    return p


def _symbol(kx, ky, g):
    return g * (WA * (4 - 2 * math.cos(kx) - 2 * math.cos(ky)) + WD * (4 - 2 * math.cos(kx + ky) - 2 * math.cos(kx - ky)))


@pytest.mark.parametrize("mx,my", [(1, 0), (0, 2), (1, 1), (3, 2), (5, -3), (12, 12)])
@pytest.mark.parametrize("cs", [0.5, 0.8])
def test_plane_waves_follow_the_discrete_dispersion_relation(oracle_mod, mx, my, cs):
    """A plane wave on a periodic 24 x 24 lattice started as an exact discrete
    mode (w^0 = cos(k.x), wdot^0 = w^0 - w^{-1}) stays one: w^n =
    cos(Omega n dt) cos(k.x) to rounding."""
    n = 24
    p = _problem(n, n, edges=("periodic",) * 4, cs=cs)
    g = cs * cs
    kx, ky = 2 * math.pi * mx / n, 2 * math.pi * my / n
    S = _symbol(kx, ky, g)
    Om = math.acos(1 - S / 2)
    x = np.arange(n)[None, :]
    y = np.arange(n)[:, None]
    prof = np.cos(kx * x + ky * y)
    o = oracle_mod.Oracle(p)
    o.set_fields(prof, (1 - math.cos(Om)) * prof)
    o.step(200)
    w, wd = o.fields()
    np.testing.assert_allclose(w, math.cos(200 * Om) * prof, rtol=0, atol=1e-10)
    o.close()


def test_stability_bound_three_quarters(oracle_mod):
    """The checkerboard mode has the largest symbol, 16 g / 3: bounded at
    g = 0.74, growing at g = 0.76."""
    n = 8
    out = {}
    for g in (0.74, 0.76):
        p = _problem(n, n, edges=("periodic",) * 4, cs=math.sqrt(g))
        prof = np.cos(np.pi * (np.arange(n)[None, :] + np.arange(n)[:, None]))
        o = oracle_mod.Oracle(p)
        c = 1 - _symbol(math.pi, math.pi, g) / 2          # cos(Omega dt); below -1 when unstable
        o.set_fields(prof, (1 - c) * prof)               # the discrete mode (exact when |c| <= 1)
        o.step(200)
        out[g] = np.abs(o.fields()[0]).max()
        o.close()
    assert out[0.74] <= 1.0 + 1e-9
    assert out[0.76] > 1e6


def _numpy_step(p, w, wd, cut_v, cut_d, wstar):
    """One D2Q9 step in the moment form: wdot' = wdot + g sum_a W_a (w_a - w),
    w' = w + dt wdot', with the value a missing link streams back: w
    (bounce-back) or 2 w* - w (anti-bounce-back), and the periodic image.
    cut_v[j, i]: link (i,j)-(i,j+1) severed; cut_d[j, i]: both diagonals of the
    cell (i..i+1, j..j+1) severed (a straight horizontal crack cuts them in
    pairs)."""
    ny, nx = w.shape
    g = p["mu"] / p["rho"] * p["dt"] ** 2 / p["dh"] ** 2
    E = p["edges"]
    per_x, per_y = E[0] == "periodic", E[2] == "periodic"
    out_w, out_wd = np.empty_like(w), np.empty_like(w)
    dirs = [(1, 0, WA), (0, 1, WA), (-1, 0, WA), (0, -1, WA), (1, 1, WD), (-1, 1, WD), (-1, -1, WD), (1, -1, WD)]
    for j in range(ny):
        for i in range(nx):
            acc = 0.0
            for dx, dy, wt in dirs:
                ni, nj = i + dx, j + dy
                # severed by the crack?
                cut = False
                if dx == 0 and dy != 0 and 0 <= nj < ny:
                    cut = cut_v[min(j, nj), i]
                elif dx != 0 and dy != 0 and 0 <= nj < ny and 0 <= ni < nx:
                    cut = cut_d[min(j, nj), min(i, ni)]
                if per_x:
                    ni %= nx
                if per_y:
                    nj %= ny
                ox, oy = not (0 <= ni < nx), not (0 <= nj < ny)
                if cut:
                    val = w[j, i]
                elif ox or oy:
                    ex = (0 if ni < 0 else 1) if ox else None
                    ey = (2 if nj < 0 else 3) if oy else None
                    if ex is not None and ey is not None:
                        e = ex if (E[ex] == "dirichlet" and E[ey] != "dirichlet") else ey
                    else:
                        e = ex if ex is not None else ey
                    val = 2 * wstar[e] - w[j, i] if E[e] == "dirichlet" else w[j, i]
                else:
                    val = w[nj, ni]
                acc += wt * (val - w[j, i])
            out_wd[j, i] = wd[j, i] + g * acc
            out_w[j, i] = w[j, i] + p["dt"] * out_wd[j, i]
    return out_w, out_wd


@pytest.mark.parametrize("edges", [("free", "free", "dirichlet", "dirichlet"), ("dirichlet", "free", "dirichlet", "free"),
                                   ("dirichlet", "dirichlet", "dirichlet", "dirichlet"),
                                   ("periodic", "periodic", "free", "dirichlet"),
                                   ("dirichlet", "free", "periodic", "periodic"), ("periodic",) * 4])
def test_one_step_against_the_moment_form(oracle_mod, edges):
    nx, ny = 9, 7
    p = _problem(nx, ny, edges)
    amps = {0: 0.3, 1: -0.7, 2: 0.45, 3: 1.1}
    p["loads"] = [{"edge": nm, "kind": "const", "amp": amps[e]}
                  for e, nm in enumerate(("left", "right", "bottom", "top")) if edges[e] == "dirichlet"]
    w0, wd0 = W.random_state(nx, ny, seed=2)
    o = oracle_mod.Oracle(p)
    o.set_fields(w0, wd0)
    o.step(1)
    w1, wd1 = o.fields()
    z = np.zeros((ny, nx), bool)
    rw, rwd = _numpy_step(p, w0, wd0, z, z, [amps[e] for e in range(4)])
    np.testing.assert_allclose(w1, rw, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wd1, rwd, rtol=0, atol=1e-14)
    o.close()


@pytest.mark.parametrize("x_start,x_tip", [(0.0, 7.3), (2.0, 6.0), (2.6, 6.9), (0.0, 12.0)])
def test_crack_links_and_bounce_back(oracle_mod, x_start, x_tip):
    """Severed links of a crack on y = jc: vertical links at x = i + 1/2 and
    both diagonals of the cell at x = i + 1, each when the point lies on the
    closed segment [x_start, x_tip]; one step with bounce-back across them."""
    nx, ny, jc = 12, 8, 4
    p = _problem(nx, ny)
    p = W.with_crack(p, mode="stationary", y=float(jc), x_start=x_start, x_tip=x_tip)
    p["loads"] = [{"edge": "top", "kind": "const", "amp": 0.2}, {"edge": "bottom", "kind": "const", "amp": -0.1}]
    o = oracle_mod.Oracle(p)
    ch, cv = o.cuts()
    d1, d2 = o.cuts_diag()
    exp_v = np.zeros((ny, nx), bool)
    exp_d = np.zeros((ny, nx), bool)
    for i in range(nx):
        exp_v[jc - 1, i] = x_start <= i + 0.5 <= x_tip
        if i + 1 < nx:
            exp_d[jc - 1, i] = x_start <= i + 1 <= x_tip
    assert not ch.any()
    np.testing.assert_array_equal(cv.astype(bool), exp_v)
    np.testing.assert_array_equal(d1.astype(bool), exp_d)
    np.testing.assert_array_equal(d2.astype(bool), exp_d)
    w0, wd0 = W.random_state(nx, ny, seed=7)
    o.set_fields(w0, wd0)
    o.step(1)
    w1, wd1 = o.fields()
    rw, rwd = _numpy_step(p, w0, wd0, exp_v, exp_d, [0.0, 0.0, -0.1, 0.2])
    np.testing.assert_allclose(w1, rw, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wd1, rwd, rtol=0, atol=1e-14)
    o.close()


def test_prescribed_growth_cuts_both_kinds_of_links(oracle_mod):
    """A two-tip crack grown at a prescribed speed: after every step the
    severed vertical and diagonal links are exactly those whose crossing
    points lie between the two ends."""
    nx, ny, jc = 40, 12, 6
    p = _problem(nx, ny)
    p = W.with_crack(p, mode="prescribed", y=float(jc), x_start=17.3, x_tip=21.8, v_rel=0.45, two_tips=True)
    p = W.with_antisymmetric_ramp(p, 1e-3, 20.0)
    o = oracle_mod.Oracle(p)
    for _ in range(100):
        o.step(1)
        lo, hi = o.left_tip_q() / 2**32, o.crack()["tip_q"] / 2**32
        _, cv = o.cuts()
        d1, d2 = o.cuts_diag()
        for i in range(nx):
            assert bool(cv[jc - 1, i]) == (lo <= i + 0.5 <= hi)
            if i + 1 < nx:
                assert bool(d1[jc - 1, i]) == bool(d2[jc - 1, i]) == (lo <= i + 1 <= hi)
    assert o.left_tip_q() == 0 and o.crack()["tip_q"] == nx * 2**32
    o.close()


def test_linear_profile_between_dirichlet_edges_is_steady(oracle_mod):
    """Anti-bounce-back with each link's own weight, on the axis and the
    diagonal links that cross a Dirichlet edge, keeps a linear profile exact.
    (The sides are periodic: at a corner with a free side the diagonal
    bounce-back returns the corner's own value where the profile has its
    neighbour's, which the one-step tests cover.)"""
    nx, ny = 10, 12
    p = _problem(nx, ny, edges=("periodic", "periodic", "dirichlet", "dirichlet"))
    a, b = 0.2, -0.03
    p["loads"] = [{"edge": "bottom", "kind": "const", "amp": a}, {"edge": "top", "kind": "const", "amp": a + b * ny}]
    y = (np.arange(ny) + 0.5)[:, None] * np.ones((1, nx))
    o = oracle_mod.Oracle(p)
    o.set_fields(a + b * y, np.zeros((ny, nx)))
    o.step(300)
    w, wd = o.fields()
    np.testing.assert_allclose(w, a + b * y, rtol=0, atol=1e-13)
    o.close()


def test_centred_crack_grows_mirror_symmetrically(oracle_mod):
    nx, ny = 96, 48
    p = _problem(nx, ny)
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_start=38.0, x_tip=58.0, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o = oracle_mod.Oracle(p)
    o.step(400)
    h, hl = o.history(), o.history_left()
    assert h["grew"].sum() > 10
    np.testing.assert_array_equal(hl["grew"], h["grew"])
    assert np.abs((nx * 2**32 - hl["tip_q"]) - h["tip_q"]).max() <= 16
    d1, d2 = o.cuts_diag()
    # mirror image of the cell column i is nx - 2 - i
    np.testing.assert_array_equal(d1[:, :-1], d1[:, :-1][:, ::-1])
    o.close()


@pytest.mark.parametrize("x_start,x_tip,v_rel", [(20.3, 40.6, 0.45), (20.0, 41.0, 0.0), (20.7, 40.2, 0.0)])
def test_macroscopic_crack_faces(oracle_mod, x_start, x_tip, v_rel):
    """The macroscopic rule on a D2Q9 crack (reading: a boundary point takes
    the normal of the crack face its severed link crosses, so x_I, x_II are
    the next two sites of its column): the boundary points are the sites of
    rows jc-1 and jc in the columns with a severed vertical link and in both
    columns of every severed diagonal pair -- which reaches a column beyond
    an end -- and after every step w_B = (3 w_I - w_II) / 2 there and
    wdot_B = (w_B - w_B(t)) / dt."""
    nx, ny, jc = 60, 20, 10
    p = _problem(nx, ny)
    p["bc_mode"] = "macroscopic"
    p = W.with_crack(p, mode="prescribed" if v_rel else "stationary", y=float(jc), x_start=x_start, x_tip=x_tip,
                     v_rel=v_rel, two_tips=bool(v_rel))
    p = W.with_antisymmetric_ramp(p, 1e-3, 30.0)
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(nx, ny, seed=4)
    o.set_fields(w0, wd0)
    cols_prev = None
    for _step in range(40):
        w_prev, _ = o.fields()
        o.step(1)
        w, wd = o.fields()
        lo = (o.left_tip_q() if v_rel else round(x_start * 2**32)) / 2**32
        hi = o.crack()["tip_q"] / 2**32
        cols = {i for i in range(nx) if lo <= i + 0.5 <= hi}
        for m in range(1, nx):
            if lo <= m <= hi:
                cols |= {m - 1, m}
        # the crack step after this LBM step may have added points: compare
        # with the set before it (the links cut up to the previous step)
        sites = set(int(k) for k in o.bpoints())
        assert {jc * nx + i for i in cols} | {(jc - 1) * nx + i for i in cols} == sites
        if cols_prev is not None:
            for i in cols_prev:
                assert w[jc, i] == pytest.approx(1.5 * w[jc + 1, i] - 0.5 * w[jc + 2, i], rel=1e-12, abs=1e-16)
                assert w[jc - 1, i] == pytest.approx(1.5 * w[jc - 2, i] - 0.5 * w[jc - 3, i], rel=1e-12, abs=1e-16)
                assert wd[jc, i] == pytest.approx(w[jc, i] - w_prev[jc, i], rel=1e-9, abs=1e-15)
        cols_prev = cols
    assert o.flags() & 2 == 0
    o.close()


def test_rejected_combinations(oracle_mod):
    with pytest.raises(Exception):
        oracle_mod.adjoint(_problem(20, 20), 2, [(5, 5)], np.zeros((2, 1)))


def test_one_step_with_the_macroscopic_edge_rule(oracle_mod):
    """D2Q9 with the macroscopic rule on the outer edges: one step is the
    nine-point moment update followed by the edge rule of Sec. 3.1 on the
    edge sites (w_B = (3 w_I - w_II)/2 on a free edge, 8/15 w*(t+dt) + 2/3 w_I
    - 1/5 w_II on a Dirichlet edge; a corner follows its Dirichlet edge, else
    the bottom / top edge), wdot_B = (w_B - w_B(t)) / dt."""
    nx, ny = 9, 8
    edges = ("dirichlet", "free", "dirichlet", "free")
    p = _problem(nx, ny, edges)
    p["bc_mode"] = "macroscopic_edges"
    amps = {0: 0.3, 2: 0.45}
    p["loads"] = [{"edge": "left", "kind": "linear", "amp": 0.3, "t": 8.0},
                  {"edge": "bottom", "kind": "linear", "amp": 0.45, "t": 8.0}]
    ws1 = [0.3 / 8.0, 0.0, 0.45 / 8.0, 0.0]          # w*(t_1)
    w0, wd0 = W.random_state(nx, ny, seed=8)
    o = oracle_mod.Oracle(p)
    o.set_fields(w0, wd0)
    o.step(1)
    w1, wd1 = o.fields()
    z = np.zeros((ny, nx), bool)
    u, _ = _numpy_step(p, w0, wd0, z, z, [0.0] * 4)   # interior values (edge sites replaced below)
    new = u.copy()

    def rule(e, a, b):
        if edges[e] == "dirichlet":
            return 8.0 / 15.0 * ws1[e] + 2.0 / 3.0 * a - 0.2 * b
        return 1.5 * a - 0.5 * b

    for j in range(1, ny - 1):
        new[j, 0] = rule(0, u[j, 1], u[j, 2])
        new[j, nx - 1] = rule(1, u[j, nx - 2], u[j, nx - 3])
    for i in range(1, nx - 1):
        new[0, i] = rule(2, u[1, i], u[2, i])
        new[ny - 1, i] = rule(3, u[ny - 2, i], u[ny - 3, i])
    new[0, 0] = rule(2, new[1, 0], new[2, 0])                       # left D, bottom D: bottom
    new[0, nx - 1] = rule(2, new[1, nx - 1], new[2, nx - 1])        # right free, bottom D: bottom
    new[ny - 1, 0] = rule(0, new[ny - 1, 1], new[ny - 1, 2])        # left D, top free: left
    new[ny - 1, nx - 1] = rule(3, new[ny - 2, nx - 1], new[ny - 3, nx - 1])   # free, free: top
    edge = np.zeros((ny, nx), bool)
    edge[0, :] = edge[-1, :] = edge[:, 0] = edge[:, -1] = True
    np.testing.assert_allclose(w1, new, rtol=0, atol=1e-14)
    np.testing.assert_allclose(wd1[edge], (new - w0)[edge], rtol=0, atol=1e-14)
    o.close()


def test_centre_crack_example_on_d2q9(oracle_mod):
    """The Sec. 5.2 configuration (quarter size) on D2Q9 with the macroscopic
    rule on every boundary: both ends grow on the first wave and stay mirror
    images; the run stays bounded."""
    p = W.kcrit_centre_crack(scale=4)
    p["lattice"] = "D2Q9"
    o = oracle_mod.Oracle(p)
    o.step(W.KCRIT_CENTRE_STEPS // 4)
    h, hl = o.history(), o.history_left()
    assert h["grew"].sum() > 5
    np.testing.assert_array_equal(hl["grew"], h["grew"])
    assert np.abs((128 * 2**32 - hl["tip_q"]) - h["tip_q"]).max() <= 16
    w, _ = o.fields()
    assert np.all(np.isfinite(w)) and np.abs(w).max() < 1.0
    assert o.flags() & 2 == 0
    o.close()
