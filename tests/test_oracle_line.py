"""Pins of the oracle's straight crack in any direction (Sec. 4.1: the crack
is a line independent of the lattice, growing along a given direction):
  * along +x it is the crack of the aligned mode, bit for bit;
  * its cut mask is exactly the set of links that the polyline of its tips
    intersects (brute force over all links, exact integer arithmetic here);
  * K from the mode III asymptotic field (eq. sif's field) around a tip at
    any angle returns that field's K;
  * transposing or mirroring the problem transposes / mirrors the fields,
    masks and tips and flips the sign of K (the criterion uses |K|);
  * a tip that meets the body's boundary stops on it, on the crack's line,
    also exactly at a corner;
  * the configurations the reading excludes are rejected."""
import copy
import math

import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

Q = 1 << 32


def _strip(nx, ny, u0=2e-3, t_ramp=60.0, edges=("free", "free", "dirichlet", "dirichlet")):
    p = W.base_problem(nx, ny, bc_mode="bounceback", edges=edges, cs=0.5)
    return W.with_antisymmetric_ramp(p, u0, t_ramp)


def _orient(a, b, c):
    v = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
    return (v > 0) - (v < 0)


def _on_box(a, b, p):
    return min(a[0], b[0]) <= p[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= p[1] <= max(a[1], b[1])


def _intersect(p1, p2, q1, q2):
    d1, d2 = _orient(q1, q2, p1), _orient(q1, q2, p2)
    d3, d4 = _orient(p1, p2, q1), _orient(p1, p2, q2)
    if d1 * d2 < 0 and d3 * d4 < 0:
        return True
    return ((d1 == 0 and _on_box(q1, q2, p1)) or (d2 == 0 and _on_box(q1, q2, p2))
            or (d3 == 0 and _on_box(p1, p2, q1)) or (d4 == 0 and _on_box(p1, p2, q2)))


def _expected_mask(nx, ny, poly):
    """Links (i,j)-(i+1,j) / (i,j)-(i,j+1) that intersect the polyline."""
    ch = np.zeros((ny, nx), np.uint8)
    cv = np.zeros((ny, nx), np.uint8)
    c = lambda i: (2 * i + 1) * (Q // 2)
    xs = [min(a[0], b[0]) for a, b in zip(poly[:-1], poly[1:])]
    for j in range(ny):
        for i in range(nx):
            for di, dj, arr in ((1, 0, ch), (0, 1, cv)):
                if i + di >= nx or j + dj >= ny:
                    continue
                a, b = (c(i), c(j)), (c(i + di), c(j + dj))
                for s0, s1 in zip(poly[:-1], poly[1:]):
                    if _intersect(a, b, s0, s1):
                        arr[j, i] = 1
                        break
    return ch, cv


def _polyline(o, p):
    cr = p["crack"]
    start = (int(np.rint(cr["x_start"] / p["dh"] * Q)), int(np.rint(cr["y_start"] / p["dh"] * Q)))
    tip0 = (int(np.rint(cr["x_tip"] / p["dh"] * Q)), int(np.rint(cr["y_tip"] / p["dh"] * Q)))
    h = o.history()
    pts = [start, tip0] + [(int(x), int(y)) for x, y in zip(h["tip_q"], h["tip_yq"])]
    out = [pts[0]]
    for q in pts[1:]:
        if q != out[-1]:
            out.append(q)
    return out


def test_along_x_is_the_aligned_crack(oracle_mod):
    p = _strip(96, 40)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 40.0)
    p1 = W.with_crack(p, mode="kcrit", y=20.0, x_start=10.0, x_tip=40.0, K_C=K_C, v_max=0.85, r0=2.0)
    p2 = W.with_line_crack(p, mode="kcrit", start=(10.0, 20.0), tip=(40.0, 20.0), K_C=K_C, v_max=0.85, r0=2.0)
    for q1, q2 in ((p1, p2), (W.with_crack(p, mode="prescribed", y=20.0, x_start=10.0, x_tip=40.0, v_rel=0.7),
                              W.with_line_crack(p, mode="prescribed", start=(10.0, 20.0), tip=(40.0, 20.0), v_rel=0.7))):
        o1, o2 = oracle_mod.Oracle(q1), oracle_mod.Oracle(q2)
        o1.step(400)
        o2.step(400)
        h1, h2 = o1.history(), o2.history()
        assert h1["grew"].sum() > 20
        np.testing.assert_array_equal(h1["tip_q"], h2["tip_q"])
        np.testing.assert_array_equal(h1["K"], h2["K"])
        assert (h2["tip_yq"] == 20 * Q).all()
        np.testing.assert_array_equal(o1.fields()[0], o2.fields()[0])
        for a, b in zip(o1.cuts(), o2.cuts()):
            np.testing.assert_array_equal(a, b)
        assert o1.flags() == o2.flags()


@pytest.mark.parametrize("start,tip,mode", [
    ((6.3, 7.1), (14.2, 11.9), "prescribed"),        # ~31 degrees
    ((30.7, 4.2), (24.9, 13.3), "prescribed"),       # ~122 degrees
    ((33.6, 29.4), (27.1, 24.6), "prescribed"),      # ~216 degrees
    ((9.2, 25.3), (17.7, 18.6), "kcrit"),            # ~-38 degrees
])
def test_mask_is_the_polyline_intersection(oracle_mod, start, tip, mode):
    nx, ny = 40, 32
    p = _strip(nx, ny, u0=3e-3, t_ramp=30.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 3e-3, float(ny))
    p = W.with_line_crack(p, mode=mode, start=start, tip=tip, v_rel=0.6, K_C=K_C, v_max=0.85, r0=1.5)
    o = oracle_mod.Oracle(p)
    o.step(120)
    h = o.history()
    assert h["grew"].sum() > 5
    poly = _polyline(o, p)
    ch, cv = _expected_mask(nx, ny, poly)
    och, ocv = o.cuts()
    np.testing.assert_array_equal(och, ch)
    np.testing.assert_array_equal(ocv, cv)
    # every advance is Delta a c rounded per component
    cx, cy = o.direction()
    L = math.hypot(tip[0] - start[0], tip[1] - start[1])
    assert abs(cx - (tip[0] - start[0]) / L) < 1e-9 and abs(cy - (tip[1] - start[1]) / L) < 1e-9
    dx, dy = np.diff(h["tip_q"]), np.diff(h["tip_yq"])
    moved = (dx != 0) | (dy != 0)
    cs, dt, dh = 0.5, p["dt"], p["dh"]
    exp = np.rint(np.outer(h["v"][1:][moved] * cs * dt / dh * Q, [cx, cy]))
    clamped = o.flags() & 1
    n_chk = moved.sum() - (1 if clamped else 0)
    np.testing.assert_array_equal(np.stack([dx[moved], dy[moved]], 1)[:n_chk], exp[:n_chk])


def _mode3_field(nx, ny, tip, theta, K, mu):
    """w = (K / mu) sqrt(2 r / pi) sin(phi / 2) around a tip at (tip) with the
    crack behind it along direction theta (phi in (-pi, pi], 0 ahead)."""
    x = np.arange(nx) + 0.5
    y = np.arange(ny) + 0.5
    X, Y = np.meshgrid(x, y)
    dx, dy = X - tip[0], Y - tip[1]
    c, s = math.cos(theta), math.sin(theta)
    u, v = dx * c + dy * s, -dx * s + dy * c          # along and left of the crack
    r = np.hypot(u, v)
    phi = np.arctan2(v, u)
    return K / mu * np.sqrt(2.0 * r / math.pi) * np.sin(phi / 2.0)


@pytest.mark.parametrize("deg", [0.0, 17.0, 30.0, 45.0, 63.0, 110.0, 200.0, 291.0])
@pytest.mark.parametrize("fit", [1.0, 3.0])
def test_K_of_the_mode3_field_at_any_angle(oracle_mod, deg, fit):
    """eq. sif on the asymptotic field itself: the pairs straddle the crack,
    so K comes back within the offset of the sites from the crack faces
    (at r >= 4 dh: a few per cent), with the field's sign."""
    nx = ny = 64
    th = math.radians(deg)
    c, s = math.cos(th), math.sin(th)
    tip = (32.0 + 0.37 * c, 32.0 + 0.37 * s + 0.011)
    start = (tip[0] - 25.0 * c, tip[1] - 25.0 * s)
    mu, K = 0.25, 3e-3
    p = W.with_line_crack(_strip(nx, ny), mode="stationary", start=start, tip=tip, r0=4.0, fit_width=fit)
    o = oracle_mod.Oracle(p)
    w = _mode3_field(nx, ny, tip, th, K, mu)
    tq = (int(np.rint(tip[0] * Q)), int(np.rint(tip[1] * Q)))
    Kf, npairs = o.evaluate_K_line(w, tq[0], tq[1], 4.0, fit)
    assert npairs >= 1
    assert abs(Kf / K - 1.0) < 0.03, (Kf / K, npairs)
    Kn, _ = o.evaluate_K_line(-w, tq[0], tq[1], 4.0, fit)
    assert Kn == -Kf


def _transposed(p):
    q = copy.deepcopy(p)
    q["nx"], q["ny"] = p["ny"], p["nx"]
    e = p["edges"]
    q["edges"] = (e[2], e[3], e[0], e[1])           # left <- bottom, right <- top, ...
    names = {"left": "bottom", "right": "top", "bottom": "left", "top": "right"}
    q["loads"] = [dict(ld, edge=names[ld["edge"]]) for ld in p["loads"]]
    cr = q["crack"]
    cr["x_start"], cr["y_start"] = p["crack"]["y_start"], p["crack"]["x_start"]
    cr["x_tip"], cr["y_tip"] = p["crack"]["y_tip"], p["crack"]["x_tip"]
    return q


@pytest.mark.parametrize("mode", ["prescribed", "kcrit"])
def test_transposed_problem(oracle_mod, mode):
    nx, ny = 48, 36
    p = _strip(nx, ny, u0=3e-3, t_ramp=30.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 3e-3, float(ny))
    p = W.with_line_crack(p, mode=mode, start=(5.2, 8.9), tip=(15.6, 14.1), v_rel=0.55, K_C=K_C, r0=1.5)
    o, t = oracle_mod.Oracle(p), oracle_mod.Oracle(_transposed(p))
    o.step(150)
    t.step(150)
    ho, ht = o.history(), t.history()
    assert ho["grew"].sum() > 5
    np.testing.assert_array_equal(ho["tip_q"], ht["tip_yq"])
    np.testing.assert_array_equal(ho["tip_yq"], ht["tip_q"])
    np.testing.assert_allclose(ht["K"], -ho["K"], rtol=1e-10, atol=1e-14)
    wo, wt = o.fields()[0], t.fields()[0]
    np.testing.assert_allclose(wt, wo.T, rtol=0, atol=1e-12 * np.abs(wo).max())
    (oh, ov), (th_, tv) = o.cuts(), t.cuts()
    np.testing.assert_array_equal(th_, ov.T)
    np.testing.assert_array_equal(tv, oh.T)


def test_mirrored_problem(oracle_mod):
    nx, ny = 48, 36
    p = _strip(nx, ny, u0=3e-3, t_ramp=30.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 3e-3, float(ny))
    p = W.with_line_crack(p, mode="kcrit", start=(4.4, 20.3), tip=(14.9, 13.2), K_C=K_C, r0=1.5)
    m = copy.deepcopy(p)
    m["loads"] = [dict(ld, edge={"bottom": "top", "top": "bottom"}.get(ld["edge"], ld["edge"])) for ld in p["loads"]]
    m["crack"]["y_start"] = ny - p["crack"]["y_start"]
    m["crack"]["y_tip"] = ny - p["crack"]["y_tip"]
    o, t = oracle_mod.Oracle(p), oracle_mod.Oracle(m)
    o.step(150)
    t.step(150)
    ho, ht = o.history(), t.history()
    assert ho["grew"].sum() > 5
    np.testing.assert_array_equal(ho["tip_q"], ht["tip_q"])
    np.testing.assert_array_equal(ny * Q - ho["tip_yq"], ht["tip_yq"])
    np.testing.assert_allclose(ht["K"], -ho["K"], rtol=1e-10, atol=1e-14)
    wo, wt = o.fields()[0], t.fields()[0]
    np.testing.assert_allclose(wt, wo[::-1], rtol=0, atol=1e-12 * np.abs(wo).max())
    (oh, ov), (th_, tv) = o.cuts(), t.cuts()
    np.testing.assert_array_equal(th_, oh[::-1])
    np.testing.assert_array_equal(tv[:-1], ov[:-1][::-1])


@pytest.mark.parametrize("start,tip,face", [
    ((4.3, 3.1), (9.6, 6.4), "right"),
    ((20.2, 3.3), (17.1, 9.8), "top"),
    ((23.2, 17.8), (17.5, 14.4), "left"),
    ((6.3, 19.6), (9.9, 12.7), "bottom"),
    ((17.75, 9.5), (22.25, 18.5), "corner"),       # slope 2 through (nx, ny) = (24, 22): no site centre on it
])
def test_tip_stops_on_the_boundary(oracle_mod, start, tip, face):
    nx, ny = 24, 22
    p = W.with_line_crack(_strip(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.8, r0=1.5)
    o = oracle_mod.Oracle(p)
    o.step(200)
    h = o.history()
    x, y = int(h["tip_q"][-1]), int(h["tip_yq"][-1])
    assert o.flags() & 1
    want = {"right": x == nx * Q, "top": y == ny * Q, "left": x == 0, "bottom": y == 0,
            "corner": (x, y) == (nx * Q, ny * Q)}[face]
    assert want, (x / Q, y / Q)
    s = (int(np.rint(start[0] * Q)), int(np.rint(start[1] * Q)))
    t0 = (int(np.rint(tip[0] * Q)), int(np.rint(tip[1] * Q)))
    # on the crack's line within the rounding of the steps
    cross = (t0[0] - s[0]) * (y - s[1]) - (t0[1] - s[1]) * (x - s[0])
    assert abs(cross) / math.hypot(t0[0] - s[0], t0[1] - s[1]) < 200 * Q * 2.0 ** -31
    # it stays there
    o.step(5)
    h2 = o.history()
    assert int(h2["tip_q"][-1]) == x and int(h2["tip_yq"][-1]) == y
    poly = _polyline(o, p)
    ch, cv = _expected_mask(nx, ny, poly)
    np.testing.assert_array_equal(o.cuts()[0], ch)
    np.testing.assert_array_equal(o.cuts()[1], cv)


@pytest.mark.parametrize("change", [
    {"start": (5.5, 5.5), "tip": (9.5, 9.5)},         # through site centres
    {"start": (3.0, 4.2), "tip": (3.0, 4.2)},         # no direction
    {"start": (-0.5, 4.2), "tip": (6.0, 5.1)},        # outside the body
    {"start": (3.0, 4.2), "tip": (6.0, 30.0)},
    {"r0": 0.5},                                      # the K window reaches the new links
    {"bc_mode": "macroscopic_edges"},
    {"lattice": "D2Q9"},
])
def test_rejected_configurations(oracle_mod, change):
    p = _strip(24, 22)
    if "bc_mode" in change:
        p["bc_mode"] = change["bc_mode"]
    if "lattice" in change:
        p["lattice"] = change["lattice"]
    p = W.with_line_crack(p, mode="prescribed", start=change.get("start", (3.0, 4.2)),
                          tip=change.get("tip", (8.0, 7.3)), v_rel=0.5, r0=change.get("r0", 2.0))
    with pytest.raises(ValueError):
        oracle_mod.Oracle(p)


# ------------------------------------------------------ both ends growing

def test_two_ends_along_x_are_the_aligned_centre_crack(oracle_mod):
    p = _strip(120, 40)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 40.0)
    for mode in ("kcrit", "prescribed"):
        q1 = W.with_crack(p, mode=mode, y=20.0, x_start=45.0, x_tip=75.0, K_C=K_C, v_rel=0.6, r0=2.0, two_tips=True)
        q2 = W.with_line_crack(p, mode=mode, start=(45.0, 20.0), tip=(75.0, 20.0), K_C=K_C, v_rel=0.6, r0=2.0,
                               two_tips=True)
        o1, o2 = oracle_mod.Oracle(q1), oracle_mod.Oracle(q2)
        o1.step(300)
        o2.step(300)
        for a, b in ((o1.history(), o2.history()), (o1.history_left(), o2.history_left())):
            assert a["grew"].sum() > 20
            np.testing.assert_array_equal(a["tip_q"], b["tip_q"])
            np.testing.assert_array_equal(a["K"], b["K"])
            assert (b["tip_yq"] == 20 * Q).all()
        np.testing.assert_array_equal(o1.fields()[0], o2.fields()[0])
        for a, b in zip(o1.cuts(), o2.cuts()):
            np.testing.assert_array_equal(a, b)


@pytest.mark.parametrize("deg", [23.0, 61.0, 137.0])
@pytest.mark.parametrize("mode", ["prescribed", "kcrit"])
def test_centre_crack_at_an_angle_is_point_symmetric(oracle_mod, deg, mode):
    """A centre crack through the middle of the body with antisymmetric loads:
    turning the body by 180 degrees about its middle maps the problem onto
    itself with w -> -w, so the two ends see the same K and move
    symmetrically, the fields satisfy w(x) = -w(R x) and the cut masks map
    onto themselves."""
    nx, ny = 64, 48
    th = math.radians(deg)
    c, s = math.cos(th), math.sin(th)
    mid = (nx / 2 + 0.013, ny / 2 + 0.007)          # no site centre on the line
    half = 6.0
    start = (mid[0] - half * c, mid[1] - half * s)
    tip = (mid[0] + half * c, mid[1] + half * s)
    # make the start the exact mirror of the tip on the grid
    tq = (int(np.rint(tip[0] * Q)), int(np.rint(tip[1] * Q)))
    start = ((nx * Q - tq[0]) / Q, (ny * Q - tq[1]) / Q)
    p = _strip(nx, ny, u0=3e-3, t_ramp=30.0)
    K_C = 0.3 * W.strip_reference_K(0.25, 3e-3, float(ny))
    p = W.with_line_crack(p, mode=mode, start=start, tip=tip, v_rel=0.5, K_C=K_C, r0=1.5, two_tips=True)
    o = oracle_mod.Oracle(p)
    o.step(120)
    hr, hl = o.history(), o.history_left()
    assert hr["grew"].sum() > 5 and hl["grew"].sum() > 5
    np.testing.assert_allclose(hl["K"], hr["K"], rtol=1e-11, atol=1e-15)
    assert np.abs(hl["tip_q"] - (nx * Q - hr["tip_q"])).max() <= 1
    assert np.abs(hl["tip_yq"] - (ny * Q - hr["tip_yq"])).max() <= 1
    w = o.fields()[0]
    np.testing.assert_allclose(w, -w[::-1, ::-1], rtol=0, atol=1e-12 * np.abs(w).max())
    ch, cv = o.cuts()
    np.testing.assert_array_equal(ch[:, :-1], ch[::-1, -2::-1])
    np.testing.assert_array_equal(cv[:-1, :], cv[-2::-1, ::-1])
    # every cut is a link that one of the two polylines meets, and back
    h_r, h_l = o.history(), o.history_left()
    s_q = (int(np.rint(start[0] * Q)), int(np.rint(start[1] * Q)))
    right = [s_q, tq] + [(int(x), int(y)) for x, y in zip(h_r["tip_q"], h_r["tip_yq"])]
    left = [tq, s_q] + [(int(x), int(y)) for x, y in zip(h_l["tip_q"], h_l["tip_yq"])]
    dedup = lambda pts: [pt for k, pt in enumerate(pts) if k == 0 or pt != pts[k - 1]]
    e1 = _expected_mask(nx, ny, dedup(right))
    e2 = _expected_mask(nx, ny, dedup(left))
    np.testing.assert_array_equal(ch, e1[0] | e2[0])
    np.testing.assert_array_equal(cv, e1[1] | e2[1])


@pytest.mark.parametrize("seed", range(6))
def test_random_lines_cut_exactly_their_polyline(oracle_mod, seed):
    """Seeded random starts, directions and lengths (one or both ends growing,
    prescribed speed): the cut mask is exactly the set of links that the
    polylines of the ends meet, every advance is Delta a c rounded per
    component, and every tip stays in the body."""
    rng = np.random.default_rng(100 + seed)
    nx, ny = int(rng.integers(20, 48)), int(rng.integers(20, 48))
    while True:
        th = rng.uniform(0.0, 2.0 * math.pi)
        L = rng.uniform(2.0, 8.0)
        sx, sy = rng.uniform(4.0, nx - 4.0), rng.uniform(4.0, ny - 4.0)
        tip = (sx + L * math.cos(th), sy + L * math.sin(th))
        if 0.5 < tip[0] < nx - 0.5 and 0.5 < tip[1] < ny - 0.5:
            break
    two = bool(seed % 2)
    p = W.with_line_crack(_strip(nx, ny), mode="prescribed", start=(sx, sy), tip=tip, v_rel=float(rng.uniform(0.3, 0.9)),
                          r0=1.5, two_tips=two)
    o = oracle_mod.Oracle(p)
    o.step(int(rng.integers(20, 80)))
    s_q = (int(np.rint(sx * Q)), int(np.rint(sy * Q)))
    t_q = (int(np.rint(tip[0] * Q)), int(np.rint(tip[1] * Q)))
    hr = o.history()
    dedup = lambda pts: [pt for k, pt in enumerate(pts) if k == 0 or pt != pts[k - 1]]
    polys = [dedup([s_q, t_q] + [(int(x), int(y)) for x, y in zip(hr["tip_q"], hr["tip_yq"])])]
    hists = [hr]
    if two:
        hl = o.history_left()
        polys.append(dedup([t_q, s_q] + [(int(x), int(y)) for x, y in zip(hl["tip_q"], hl["tip_yq"])]))
        hists.append(hl)
    ch = np.zeros((ny, nx), np.uint8)
    cv = np.zeros((ny, nx), np.uint8)
    for poly in polys:
        a, b = _expected_mask(nx, ny, poly)
        ch |= a
        cv |= b
    och, ocv = o.cuts()
    np.testing.assert_array_equal(och, ch)
    np.testing.assert_array_equal(ocv, cv)
    cx, cy = o.direction()
    q = p["crack"]["v_rel"] * 0.5 * p["dt"] / p["dh"] * Q
    for h, sign in zip(hists, (1, -1)):
        x, y = np.asarray(h["tip_q"]), np.asarray(h["tip_yq"])
        assert (x >= 0).all() and (x <= nx * Q).all() and (y >= 0).all() and (y <= ny * Q).all()
        dx, dy = np.diff(x), np.diff(y)
        free = (x[1:] > 0) & (x[1:] < nx * Q) & (y[1:] > 0) & (y[1:] < ny * Q)
        np.testing.assert_array_equal(dx[free], sign * np.rint(q * cx) * np.ones(free.sum()))
        np.testing.assert_array_equal(dy[free], sign * np.rint(q * cy) * np.ones(free.sum()))


def test_benchmark_line_workload_grows(oracle_mod):
    """The benchmark's crack at 20 degrees (kcrit_line) at 1/16 scale: the
    K-criterion starts the growth during the ramp and the tip keeps to the
    crack's line until it stops on the top edge."""
    p = W.kcrit_line(scale=16)
    o = oracle_mod.Oracle(p)
    o.step(3000)
    h = o.history()
    first = int(np.argmax(h["v"] > 0))
    assert 0 < first < 5000 // 16
    cr = p["crack"]
    s_q = (cr["x_start"] * Q, cr["y_start"] * Q)
    c = (math.cos(math.radians(20.0)), math.sin(math.radians(20.0)))
    off = -(h["tip_q"] - s_q[0]) * c[1] + (h["tip_yq"] - s_q[1]) * c[0]
    assert np.abs(off).max() < 1e-6 * Q
    assert o.flags() & 1 and int(h["tip_yq"][-1]) == p["ny"] * Q


# ------------------------------------------ the macroscopic rule (oracle only)

@pytest.mark.parametrize("two", [False, True])
def test_macroscopic_along_x_is_the_aligned_rule(oracle_mod, two):
    """With c = (1, 0) every x_I, x_II is a site and the line's normal is the
    face's: the rule of the aligned crack, bit for bit."""
    p = W.base_problem(120, 48, bc_mode="macroscopic", edges=("free", "free", "dirichlet", "dirichlet"), cs=0.5)
    p = W.with_antisymmetric_ramp(p, 2e-3, 60.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    q1 = W.with_crack(p, mode="kcrit", y=24.0, x_start=45.0, x_tip=70.0, K_C=K_C, r0=2.0, two_tips=two)
    q2 = W.with_line_crack(p, mode="kcrit", start=(45.0, 24.0), tip=(70.0, 24.0), K_C=K_C, r0=2.0, two_tips=two)
    o1, o2 = oracle_mod.Oracle(q1), oracle_mod.Oracle(q2)
    o1.step(250)
    o2.step(250)
    h1, h2 = o1.history(), o2.history()
    assert h1["grew"].sum() > 10
    np.testing.assert_array_equal(h1["tip_q"], h2["tip_q"])
    np.testing.assert_array_equal(h1["K"], h2["K"])
    np.testing.assert_array_equal(o1.fields()[0], o2.fields()[0])
    np.testing.assert_array_equal(np.sort(o1.bpoints()), np.sort(o2.bpoints()))
    assert o1.flags() == o2.flags() and not o1.flags() & 2


@pytest.mark.parametrize("deg", [17.0, 45.0, 71.0, 143.0])
def test_macroscopic_keeps_a_field_linear_along_the_crack(oracle_mod, deg):
    """w = a t (t the distance along c) has no normal derivative on the crack
    faces and is harmonic: after one step from it (with wdot = 0), every
    boundary point of the rule holds a t(x_B) -- the quadratic's zero slope,
    the distances s_B, s_I, s_II and the one-sided bilinear stencils all
    have to be right for that."""
    nx = ny = 64
    th = math.radians(deg)
    c, s = math.cos(th), math.sin(th)
    mid = (32.013, 32.007)
    start, tip = (mid[0] - 12 * c, mid[1] - 12 * s), (mid[0] + 12 * c, mid[1] + 12 * s)
    p = W.base_problem(nx, ny, bc_mode="macroscopic", edges=("free",) * 4, cs=0.5)
    p["loads"] = []
    p = W.with_line_crack(p, mode="stationary", start=start, tip=tip, r0=2.0)
    o = oracle_mod.Oracle(p)
    cx, cy = o.direction()
    sx, sy = np.rint(start[0] * Q) / Q, np.rint(start[1] * Q) / Q
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    a = 1e-3
    w0 = a * ((X - sx) * cx + (Y - sy) * cy)
    o.set_fields(w0, np.zeros_like(w0))
    o.step(1)
    bp = o.bpoints()
    assert len(bp) > 20
    w = o.fields()[0].ravel()
    np.testing.assert_allclose(w[bp], w0.ravel()[bp], rtol=0, atol=1e-14)
    assert o.flags() == 0


def test_macroscopic_inclined_growth_stays_finite(oracle_mod):
    """K-criterion growth at 30 degrees with the rule on the crack faces:
    the run stays finite and grows (the rule's stability for this reading),
    up to the step before the tip comes within reach of the top edge, where
    the stencils of the points it creates would leave the body (flagged)."""
    nx, ny = 96, 64
    p = W.base_problem(nx, ny, bc_mode="macroscopic", edges=("free", "free", "dirichlet", "dirichlet"), cs=0.5)
    p = W.with_antisymmetric_ramp(p, 3e-3, 40.0)
    K_C = 0.3 * W.strip_reference_K(0.25, 3e-3, float(ny))
    th = math.radians(30.0)
    start = (20.3, 24.1)
    tip = (start[0] + 15 * math.cos(th), start[1] + 15 * math.sin(th))
    p = W.with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, r0=2.0)
    o = oracle_mod.Oracle(p)
    o.step(200)
    h = o.history()
    w = o.fields()[0]
    assert np.isfinite(w).all() and np.abs(w).max() < 10 * 3e-3
    assert (h["v"] > 0).sum() > 100
    assert o.flags() == 0
    o.step(100)                     # the tip reaches the top edge
    assert o.flags() & 1 and o.flags() & 2


@pytest.mark.parametrize("deg", [17.0, 45.0, 71.0, 143.0])
def test_macroscopic_keeps_a_jump_across_the_crack(oracle_mod, deg):
    """w = a t + g sign(d) (d the signed distance from the crack's line): on
    each side linear along the crack, with a jump across it -- a stencil that
    reached across the crack would mix the two sides.  After one step every
    boundary point holds its own side's value."""
    nx = ny = 64
    th = math.radians(deg)
    c, s = math.cos(th), math.sin(th)
    mid = (32.013, 32.007)
    start, tip = (mid[0] - 12 * c, mid[1] - 12 * s), (mid[0] + 12 * c, mid[1] + 12 * s)
    p = W.base_problem(nx, ny, bc_mode="macroscopic", edges=("free",) * 4, cs=0.5)
    p["loads"] = []
    p = W.with_line_crack(p, mode="stationary", start=start, tip=tip, r0=2.0)
    o = oracle_mod.Oracle(p)
    cx, cy = o.direction()
    sx, sy = np.rint(start[0] * Q) / Q, np.rint(start[1] * Q) / Q
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    t = (X - sx) * cx + (Y - sy) * cy
    d = -(X - sx) * cy + (Y - sy) * cx
    w0 = 1e-3 * t + 2e-3 * np.sign(d)
    o.set_fields(w0, np.zeros_like(w0))
    o.step(1)
    bp = o.bpoints()
    # the boundary points beside the crack's inner stretch (the ends' points
    # see the field wrap around the tip, where it is no longer a solution)
    inner = bp[(t.ravel()[bp] > 3.0) & (t.ravel()[bp] < 21.0)]
    assert len(inner) > 20
    w = o.fields()[0].ravel()
    np.testing.assert_allclose(w[inner], w0.ravel()[inner], rtol=0, atol=1e-14)


def test_macroscopic_stencils_reach_only_away_from_the_line():
    """The geometry the face solve rests on (Sec. 3.1 read for a crack off the
    lattice's axes): every corner with weight of the x_I = x_B + n and
    x_II = x_B + 2n cells lies strictly farther from the line than x_B, on
    its side, except x_B's own site in the x_I cell, whose weight in w_B
    stays below 0.2; so the points' coupling is acyclic apart from that term."""
    rng = np.random.default_rng(7)
    for _ in range(400):
        th = rng.uniform(0.0, 2 * np.pi)
        c = np.array([np.cos(th), np.sin(th)])
        if min(abs(c[0]), abs(c[1])) < 1e-3:
            continue
        s0 = rng.uniform(0.0, 1.0, 2)
        for i in range(-3, 4):
            for j in range(-3, 4):
                b = np.array([i + 0.5, j + 0.5])
                d = -(b[0] - s0[0]) * c[1] + (b[1] - s0[1]) * c[0]
                if not (0.0 < abs(d) < 1.5):
                    continue
                n = np.sign(d) * np.array([-c[1], c[0]])
                sB, sI, sII = abs(d), abs(d) + 1.0, abs(d) + 2.0
                qq = (sB ** 2 - sI ** 2) / (sII ** 2 - sI ** 2)
                for m, coef in ((1, 1.0 - qq), (2, qq)):
                    g = b + m * n - 0.5
                    i0, j0 = np.floor(g).astype(int)
                    t = g - np.array([i0, j0])
                    for di in (0, 1):
                        for dj in (0, 1):
                            wgt = (t[0] if di else 1 - t[0]) * (t[1] if dj else 1 - t[1])
                            if wgt == 0.0:
                                continue
                            k = np.array([i0 + di + 0.5, j0 + dj + 0.5])
                            dk = -(k[0] - s0[0]) * c[1] + (k[1] - s0[1]) * c[0]
                            assert np.sign(dk) == np.sign(d)
                            if np.allclose(k, b):
                                assert m == 1 and 0.0 < coef * wgt < 0.2
                            else:
                                assert abs(dk) > abs(d) + 1e-9
