"""A straight crack in any direction (lbm_create_line, Sec. 4.1) through the
C ABI against the oracle: FP64 fields within 1e-12 and FP32 within 1e-5 of
the state's scale, tips (x and y) and both cut masks bit-exact, K within
1e-9 (FP64) / 0.5 % (FP32) of its largest value; angles in all four
quadrants, lattices spanning several column blocks and row bands with
ragged ends, every edge kind, prescribed and K-criterion growth, stops on
each face of the body and at a corner, single launches and graph chunks,
the deferred crack step read between chunks, reset and checkpoint resume,
and the calls that reject the handle."""
import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}
Q = 1 << 32


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_12412_gb300 import lbm
    lbm.load_library()
    return lbm


def _problem(nx, ny, edges=("free", "free", "dirichlet", "dirichlet"), u0=3e-3, t_ramp=40.0):
    p = W.base_problem(nx, ny, bc_mode="bounceback", edges=edges, cs=0.5)
    names = ("left", "right", "bottom", "top")
    sign = {"left": -1.0, "right": 1.0, "bottom": -1.0, "top": 1.0}
    p["loads"] = [{"edge": names[e], "kind": "linear", "amp": sign[names[e]] * u0, "t": t_ramp}
                  for e in range(4) if edges[e] == "dirichlet"]
    return p


def _run(oracle_mod, gpu, p, storage, chunks, solve=None):
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, storage)
    if solve is not None:
        # the macroscopic faces' solve: 0 chunked (where the coupling allows), 1 one CTA
        g.chunked = g.set_face_solve(solve)
    for n in chunks:
        o.step(n)
        g.step(n)
    return o, g


def _close(o, g, tol):
    wo, wdo = o.fields()
    wg, wdg = g.fields()
    scale = max(np.abs(wo).max(), 1e-300)
    assert np.abs(wg - wo).max() <= tol * scale, np.abs(wg - wo).max() / scale
    assert np.abs(wdg - wdo).max() <= tol * scale, np.abs(wdg - wdo).max() / scale


def _masks(o, g):
    ch, cv = o.cuts()
    np.testing.assert_array_equal(g.cut_mask("h"), ch.astype(bool))
    np.testing.assert_array_equal(g.cut_mask("v"), cv.astype(bool))


def _tips(o, g, n):
    ho, hg = o.history(), g.history(cap=n)
    np.testing.assert_array_equal(hg["tip_q"], ho["tip_q"][-len(hg["tip_q"]):])
    np.testing.assert_array_equal(hg["tip_yq"], ho["tip_yq"][-len(hg["tip_yq"]):])
    np.testing.assert_array_equal(hg["npairs"], ho["npairs"][-len(hg["npairs"]):])
    return ho, hg


ANGLES = [  # (start, tip) on a 300 x 90 lattice: ~17, ~122, ~200 and ~-40 degrees
    ((20.3, 30.7), (120.9, 61.2)),
    ((230.4, 8.3), (200.1, 56.8)),
    ((285.6, 70.2), (170.7, 28.4)),
    ((15.7, 80.9), (80.2, 26.6)),
]


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("start,tip", ANGLES)
def test_prescribed_growth_against_oracle(oracle_mod, gpu, storage, start, tip):
    nx, ny = 300 if storage == "f64" else 700, 90
    sx = 1.0 if storage == "f64" else 700.0 / 300.0
    p = _problem(nx, ny)
    p = W.with_line_crack(p, mode="prescribed", start=(start[0] * sx, start[1]), tip=(tip[0] * sx, tip[1]),
                          v_rel=0.7, r0=2.0, fit_width=2.0)
    o, g = _run(oracle_mod, gpu, p, storage, [7, 64, 29, 100])
    _close(o, g, TOL[storage])
    _masks(o, g)
    ho, hg = _tips(o, g, 200)
    assert (np.diff(ho["tip_q"]) != 0).sum() > 50
    np.testing.assert_allclose(hg["K"], ho["K"], rtol=0, atol=(1e-9 if storage == "f64" else 5e-3) * np.abs(ho["K"]).max())
    st = g.crack_state()
    assert st["n_cut"] == int(o.cuts()[0].sum() + o.cuts()[1].sum())
    assert g.tip_q() == (int(ho["tip_q"][-1]), int(ho["tip_yq"][-1]))


@pytest.mark.parametrize("start,tip", ANGLES[:2])
def test_kcrit_growth_fp64(oracle_mod, gpu, start, tip):
    p = _problem(300, 90, u0=4e-3, t_ramp=60.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 4e-3, 90.0)
    p = W.with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, v_max=0.85, r0=2.0)
    o, g = _run(oracle_mod, gpu, p, "f64", [150, 150])
    ho, hg = _tips(o, g, 300)
    assert (ho["v"] > 0).sum() > 10
    np.testing.assert_allclose(hg["K"], ho["K"], rtol=0, atol=1e-9 * np.abs(ho["K"]).max())
    _masks(o, g)
    _close(o, g, TOL["f64"])


def test_kcrit_growth_fp32_tolerance(oracle_mod, gpu):
    """FP32 fields with an FP64 K decision: the tip follows the oracle's within
    one spacing and the growth count within a few steps."""
    p = _problem(300, 90, u0=4e-3, t_ramp=60.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 4e-3, 90.0)
    p = W.with_line_crack(p, mode="kcrit", start=ANGLES[0][0], tip=ANGLES[0][1], K_C=K_C, v_max=0.85, r0=2.0)
    o, g = _run(oracle_mod, gpu, p, "f32", [300])
    ho, hg = o.history(), g.history(cap=300)
    assert (ho["v"] > 0).sum() > 10
    assert np.abs(hg["tip_q"] - ho["tip_q"]).max() < Q and np.abs(hg["tip_yq"] - ho["tip_yq"]).max() < Q
    assert abs(int((hg["v"] > 0).sum()) - int((ho["v"] > 0).sum())) <= 3


@pytest.mark.parametrize("edges", [("dirichlet", "free", "dirichlet", "free"), ("periodic", "periodic", "free", "dirichlet"),
                                   ("dirichlet", "dirichlet", "periodic", "periodic"), ("free",) * 4])
@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_edge_kinds(oracle_mod, gpu, edges, storage):
    p = _problem(261, 70, edges=edges)
    if edges == ("free",) * 4:
        p["loads"] = []
        init = W.random_state(261, 70, seed=5, dtype=np.float64 if storage == "f64" else np.float32)
    else:
        init = None
    p = W.with_line_crack(p, mode="prescribed", start=(40.2, 12.6), tip=(90.9, 40.3), v_rel=0.8, r0=1.5)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, storage)
    if init is not None:
        o.set_fields(*init)
        g.set_fields(*init)
    for n in (5, 64, 61):
        o.step(n)
        g.step(n)
    _close(o, g, TOL[storage])
    _masks(o, g)
    _tips(o, g, 130)


@pytest.mark.parametrize("start,tip,face", [
    ((4.3, 3.1), (9.6, 6.4), "right"),
    ((20.2, 3.3), (17.1, 9.8), "top"),
    ((23.2, 17.8), (17.5, 14.4), "left"),
    ((6.3, 19.6), (9.9, 12.7), "bottom"),
    ((17.75, 9.5), (22.25, 18.5), "corner"),
])
def test_tip_stops_on_the_boundary(oracle_mod, gpu, start, tip, face):
    nx, ny = 24, 22
    p = W.with_line_crack(_problem(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.8, r0=1.5)
    o, g = _run(oracle_mod, gpu, p, "f64", [100, 5])
    ho, hg = _tips(o, g, 105)
    assert g.crack_state()["flags"] & 1
    x, y = g.tip_q()
    assert {"right": x == nx * Q, "top": y == ny * Q, "left": x == 0, "bottom": y == 0,
            "corner": (x, y) == (nx * Q, ny * Q)}[face]
    _masks(o, g)
    _close(o, g, TOL["f64"])


def test_along_x_matches_the_aligned_crack(oracle_mod, gpu):
    """A line crack along +x on the GPU against the oracle's aligned crack."""
    p = _problem(300, 90)
    pa = W.with_crack(p, mode="prescribed", y=45.0, x_start=10.0, x_tip=60.0, v_rel=0.7)
    pl = W.with_line_crack(p, mode="prescribed", start=(10.0, 45.0), tip=(60.0, 45.0), v_rel=0.7)
    o = oracle_mod.Oracle(pa)
    g = gpu.Lattice(pl, "f64")
    o.step(200)
    g.step(200)
    _close(o, g, TOL["f64"])
    np.testing.assert_array_equal(g.history(cap=200)["tip_q"], o.history()["tip_q"])
    _masks(o, g)


def test_reset_and_checkpoint(oracle_mod, gpu, tmp_path):
    p = W.with_line_crack(_problem(300, 90), mode="prescribed", start=ANGLES[1][0], tip=ANGLES[1][1], v_rel=0.6)
    g = gpu.Lattice(p, "f64")
    g.step(70)
    path = str(tmp_path / "line.lbm")
    g.save(path)
    g.step(90)
    w1, wd1 = g.fields()
    m1 = (g.cut_mask("h"), g.cut_mask("v"))
    t1 = g.tip_q()
    g.load(path)
    g.step(90)
    w2, wd2 = g.fields()
    np.testing.assert_array_equal(w1, w2)
    np.testing.assert_array_equal(wd1, wd2)
    assert g.tip_q() == t1
    np.testing.assert_array_equal(m1[0], g.cut_mask("h"))
    np.testing.assert_array_equal(m1[1], g.cut_mask("v"))
    g.reset()
    g.step(160)
    np.testing.assert_array_equal(g.fields()[0], w1)
    assert g.tip_q() == t1
    o = oracle_mod.Oracle(p)
    o.step(160)
    _masks(o, g)


@pytest.mark.parametrize("mode", ["kcrit", "prescribed"])
def test_full_size_in_the_benchmark_shape(oracle_mod, gpu, mode):
    """4096 x 2048 FP32, the benchmark's crack at 20 degrees (and the same
    crack growing at a prescribed speed), in the launch shape the benchmark
    times: every output after 12 steps from a seeded state."""
    p = W.kcrit_line()
    if mode == "prescribed":
        p["crack"] = dict(p["crack"], mode="prescribed", v_rel=0.8)
    init = W.random_state(p["nx"], p["ny"], seed=23, dtype=np.float32)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f32")
    o.set_fields(*init)
    g.set_fields(*init)
    o.step(12)
    g.step(12)
    _close(o, g, TOL["f32"])
    _masks(o, g)
    ho, hg = o.history(), g.history(cap=12)
    np.testing.assert_array_equal(hg["npairs"], ho["npairs"])
    np.testing.assert_allclose(hg["K"], ho["K"], rtol=0, atol=5e-3 * np.abs(ho["K"]).max())
    if mode == "prescribed":
        np.testing.assert_array_equal(hg["tip_q"], ho["tip_q"])
        np.testing.assert_array_equal(hg["tip_yq"], ho["tip_yq"])
        assert (np.diff(ho["tip_q"]) != 0).all()


def test_calls_that_reject_the_handle(gpu):
    p = W.with_line_crack(_problem(64, 32), mode="prescribed", start=(3.3, 4.1), tip=(9.2, 7.7), v_rel=0.5)
    g = gpu.Lattice(p, "f32")
    with pytest.raises(gpu.LbmError) as ei:
        g.crack_state_left()
    assert ei.value.status == gpu.A.LBM_ERR_STATE
    straight = gpu.Lattice(W.prescribed_strip(64, 32, 0.4), "f32")
    with pytest.raises(gpu.LbmError):
        gpu.Batch([g, straight])       # cracks along +x and in any direction apart
    straight.close()
    b = gpu.Batch([g])
    with pytest.raises(gpu.LbmError):
        b.set_shape(64, 16)
    with pytest.raises(gpu.LbmError):
        b.set_persistent(True)
    b.close()
    launch = gpu.lbm_get_launch(g.h)
    assert launch["ctas"] == 1 + -(-64 // 512) * -(-32 // launch["band_rows"])
    q = gpu.Lattice(W.plain_fp64(), "f64")
    with pytest.raises(gpu.LbmError) as ei:
        gpu.lbm_line_tip(q.h)
    assert ei.value.status == gpu.A.LBM_ERR_STATE


# directions where the band's description changes form: along the axes (one
# component of c is 0), near them, and at 45 degrees (the switch between the
# per-column and per-row descriptions)
AXES = [
    ((30.0, 61.3), (90.0, 61.3)),        # +x on a half row (the line crack's own code path)
    ((250.0, 40.6), (200.0, 40.6)),      # -x
    ((120.3, 10.0), (120.3, 60.0)),      # +y
    ((150.6, 190.0), (150.6, 140.0)),    # -y
    ((40.0, 20.3), (100.0, 80.3)),       # 45 degrees
    ((260.0, 30.7), (200.0, 90.7)),      # 135 degrees
    ((20.0, 100.2), (120.0, 100.72)),    # 0.3 degrees
    ((170.2, 15.0), (170.72, 115.0)),    # 89.7 degrees
]


@pytest.mark.parametrize("start,tip", AXES)
def test_directions_near_the_axes(oracle_mod, gpu, start, tip):
    p = W.with_line_crack(_problem(300, 200), mode="prescribed", start=start, tip=tip, v_rel=0.7, r0=2.0)
    o, g = _run(oracle_mod, gpu, p, "f32", [64, 86])
    _close(o, g, TOL["f32"])
    _masks(o, g)
    ho, hg = _tips(o, g, 150)
    assert (np.diff(ho["tip_q"]) != 0).sum() + (np.diff(ho["tip_yq"]) != 0).sum() > 50


# ------------------------------------------------------ both ends growing

def _centre(nx, ny, deg, half):
    """A centre crack through the middle of the body at `deg` degrees, its
    start the exact mirror of its tip on the grid."""
    th = np.radians(deg)
    mid = (nx / 2 + 0.013, ny / 2 + 0.007)
    tip = (mid[0] + half * np.cos(th), mid[1] + half * np.sin(th))
    tq = (int(np.rint(tip[0] * Q)), int(np.rint(tip[1] * Q)))
    return ((nx * Q - tq[0]) / Q, (ny * Q - tq[1]) / Q), tip


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("deg", [23.0, 61.0, 137.0, 200.0])
def test_two_ends_prescribed(oracle_mod, gpu, storage, deg):
    nx, ny = (300, 200) if storage == "f64" else (700, 200)
    start, tip = _centre(nx, ny, deg, 20.0)
    p = W.with_line_crack(_problem(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0,
                          two_tips=True)
    o, g = _run(oracle_mod, gpu, p, storage, [7, 64, 49])
    _close(o, g, TOL[storage])
    _masks(o, g)
    _tips(o, g, 120)
    hl_o, hl_g = o.history_left(), g.history_left(cap=120)
    np.testing.assert_array_equal(hl_g["tip_q"], hl_o["tip_q"])
    np.testing.assert_array_equal(hl_g["tip_yq"], hl_o["tip_yq"])
    np.testing.assert_array_equal(hl_g["npairs"], hl_o["npairs"])
    assert (np.diff(hl_o["tip_q"]) != 0).sum() + (np.diff(hl_o["tip_yq"]) != 0).sum() > 50
    assert g.tip_q_left() == (int(hl_o["tip_q"][-1]), int(hl_o["tip_yq"][-1]))


@pytest.mark.parametrize("deg", [23.0, 137.0])
def test_two_ends_kcrit_fp64(oracle_mod, gpu, deg):
    nx, ny = 300, 200
    start, tip = _centre(nx, ny, deg, 25.0)
    p = _problem(nx, ny, u0=4e-3, t_ramp=60.0)
    K_C = 0.3 * W.strip_reference_K(0.25, 4e-3, float(ny))
    p = W.with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o, g = _run(oracle_mod, gpu, p, "f64", [150, 150])
    ho, hg = _tips(o, g, 300)
    hlo, hlg = o.history_left(), g.history_left(cap=300)
    assert (ho["v"] > 0).sum() > 10 and (hlo["v"] > 0).sum() > 10
    np.testing.assert_array_equal(hlg["tip_q"], hlo["tip_q"])
    np.testing.assert_array_equal(hlg["tip_yq"], hlo["tip_yq"])
    np.testing.assert_allclose(hlg["K"], hlo["K"], rtol=0, atol=1e-9 * np.abs(hlo["K"]).max())
    _masks(o, g)
    _close(o, g, TOL["f64"])


def test_two_ends_along_x_match_the_aligned_centre_crack(oracle_mod, gpu):
    p = _problem(300, 90)
    pa = W.with_crack(p, mode="prescribed", y=45.0, x_start=130.0, x_tip=170.0, v_rel=0.7, two_tips=True)
    pl = W.with_line_crack(p, mode="prescribed", start=(130.0, 45.0), tip=(170.0, 45.0), v_rel=0.7, two_tips=True)
    o = oracle_mod.Oracle(pa)
    g = gpu.Lattice(pl, "f64")
    o.step(200)
    g.step(200)
    _close(o, g, TOL["f64"])
    np.testing.assert_array_equal(g.history(cap=200)["tip_q"], o.history()["tip_q"])
    np.testing.assert_array_equal(g.history_left(cap=200)["tip_q"], o.history_left()["tip_q"])
    _masks(o, g)


def test_two_ends_stop_on_the_boundary_and_resume(oracle_mod, gpu, tmp_path):
    """Both ends run into the body's boundary; a checkpoint taken on the way
    resumes bit-identically, records included."""
    nx, ny = 40, 30
    p = W.with_line_crack(_problem(nx, ny), mode="prescribed", start=(17.3, 12.1), tip=(23.9, 16.6), v_rel=0.8,
                          r0=1.5, two_tips=True)
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f64")
    o.step(20)
    g.step(20)
    path = str(tmp_path / "two.lbm")
    g.save(path)
    o.step(80)
    g.step(80)
    assert g.crack_state()["flags"] & 1 and g.crack_state_left()["flags"] & 1
    _masks(o, g)
    _close(o, g, TOL["f64"])
    h1, l1 = g.history(cap=100), g.history_left(cap=100)
    np.testing.assert_array_equal(l1["tip_yq"], o.history_left()["tip_yq"])
    g.load(path)
    g.step(80)
    h2, l2 = g.history(cap=100), g.history_left(cap=100)
    for a, b in ((h1, h2), (l1, l2)):
        for k in ("tip_q", "tip_yq", "K"):
            np.testing.assert_array_equal(a[k], b[k])


# w of the 16-bit wdot forms: the bounds of test_gpu_mixed.py (stored wdot
# rounded to 8 / 11 significant bits every step; not a parity bar)
BOUND_16 = {"f32_bf16": 1e-2, "f32_f16": 1e-3}


@pytest.mark.parametrize("storage", ["f32_bf16", "f32_f16"])
@pytest.mark.parametrize("two", [False, True])
def test_sixteen_bit_wdot(oracle_mod, gpu, storage, two):
    nx, ny = 700, 200
    start, tip = _centre(nx, ny, 33.0, 20.0)
    p = W.with_line_crack(_problem(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0, two_tips=two)
    o, g = _run(oracle_mod, gpu, p, storage, [64, 86])
    wo, _ = o.fields()
    wg, _ = g.fields()
    assert np.abs(wg - wo).max() < BOUND_16[storage] * np.abs(wo).max()
    _masks(o, g)
    _tips(o, g, 150)


# ------------------------------------------ the macroscopic rule on the faces

def _macro(nx, ny, u0=3e-3, t_ramp=40.0):
    p = _problem(nx, ny, u0=u0, t_ramp=t_ramp)
    p["bc_mode"] = "macroscopic"
    return p


@pytest.mark.parametrize("solve", [0, 1])
@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("deg,two", [(23.0, False), (137.0, False), (61.0, True), (2.0, True), (0.5, True)])
def test_macroscopic_faces_prescribed(oracle_mod, gpu, storage, deg, two, solve):
    """Both solves of the faces' system: the chunked one (a CTA per stretch of
    the line, level by level; at 0.5 degrees the coupling is deeper than it
    takes, so the one-CTA solve runs) and the one-CTA Jacobi solve."""
    nx, ny = 300, 200
    start, tip = _centre(nx, ny, deg, 20.0)
    p = W.with_line_crack(_macro(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0, two_tips=two)
    # 70 steps: the solve along these lines meets its bitwise fixpoint
    # throughout (the oracle flags a solve that ends without one)
    o, g = _run(oracle_mod, gpu, p, storage, [7, 40, 23], solve=solve)
    assert g.chunked == (solve == 0 and deg != 0.5)
    assert o.flags() == 0 and g.crack_state()["flags"] == 0
    _close(o, g, TOL[storage])
    _masks(o, g)
    _tips(o, g, 70)


def test_macroscopic_faces_kcrit_fp64(oracle_mod, gpu):
    nx, ny = 160, 48
    start, tip = _centre(nx, ny, 23.0, 10.0)
    p = _macro(nx, ny, u0=4e-3, t_ramp=10.0)
    K_C = 0.2 * W.strip_reference_K(0.25, 4e-3, float(ny))
    p = W.with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    o, g = _run(oracle_mod, gpu, p, "f64", [60, 80], solve=0)
    assert o.flags() == 0 and g.chunked
    ho, hg = _tips(o, g, 140)
    assert (ho["v"] > 0).sum() > 10 and (o.history_left()["v"] > 0).sum() > 10
    np.testing.assert_allclose(hg["K"], ho["K"], rtol=0, atol=1e-9 * np.abs(ho["K"]).max())
    _masks(o, g)
    _close(o, g, TOL["f64"])


def test_macroscopic_faces_beyond_the_kernels_shared_memory(oracle_mod, gpu):
    """A centre crack long enough that its boundary points outnumber the face
    solve's shared memory (3008 points), so the sweeps run in its scratch."""
    nx, ny = 1800, 300
    start, tip = _centre(nx, ny, 8.0, 860.0)
    p = W.with_line_crack(_macro(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.5, r0=2.0, two_tips=True)
    o, g = _run(oracle_mod, gpu, p, "f64", [5, 7], solve=1)
    assert len(o.bpoints()) > 3008
    assert o.flags() == 0
    _close(o, g, TOL["f64"])
    _masks(o, g)
    _tips(o, g, 12)


@pytest.mark.parametrize("solve", [0, 1])
def test_unsupported_face_points_are_flagged_like_the_oracle(oracle_mod, gpu, solve):
    """A crack with macroscopic faces that grows to within two spacings of an
    edge: a new boundary point whose x_I or x_II cell reaches outside the
    body is not supported by the rule; the oracle flags it when it adds the
    point (at step n_f), the GPU when its face solve first uses the point
    (the next step).  Both report FLAG_UNSUPPORTED = 2 from then on, neither
    before; the fields agree until then."""
    import math
    nx, ny = 160, 60
    start, ang = (60.3, 30.2), math.radians(23.0)
    tip = (start[0] + 20 * math.cos(ang), start[1] + 20 * math.sin(ang))
    p = W.with_line_crack(_macro(nx, ny), mode="prescribed", start=start, tip=tip, v_rel=0.7, r0=2.0, two_tips=False)
    o = oracle_mod.Oracle(p)
    n_f = 0
    while not o.flags() & 2:
        o.step(1)
        n_f += 1
        assert n_f < 400
    assert 100 < n_f
    o.close()
    o = oracle_mod.Oracle(p)
    g = gpu.Lattice(p, "f64")
    g.set_face_solve(solve)
    o.step(n_f - 2)
    g.step(n_f - 2)
    assert o.flags() == 0 and g.crack_state()["flags"] == 0
    _close(o, g, TOL["f64"])
    _masks(o, g)
    o.step(4)
    g.step(4)
    assert o.flags() & 2 and g.crack_state()["flags"] & 2
    o.close()
    g.close()


# ------------------------------------------------------------------ batches

def _line_batch_problems():
    """Uneven lattices with cracks in any direction: the four quadrant angles
    (prescribed), K-criterion growth, both ends of a centre crack, and the
    macroscopic rule on the faces (one and two ends), on lattices of one to
    two column blocks with ragged ends."""
    ps = []
    for start, tip in ANGLES:
        ps.append(W.with_line_crack(_problem(300, 90), mode="prescribed", start=start, tip=tip, v_rel=0.7, r0=2.0,
                                    fit_width=2.0))
    q = _problem(300, 90, u0=4e-3, t_ramp=60.0)
    K_C = 0.4 * W.strip_reference_K(0.25, 4e-3, 90.0)
    ps.append(W.with_line_crack(q, mode="kcrit", start=ANGLES[0][0], tip=ANGLES[0][1], K_C=K_C, v_max=0.85, r0=2.0))
    start, tip = _centre(300, 200, 137.0, 20.0)
    ps.append(W.with_line_crack(_problem(300, 200), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0,
                                two_tips=True))
    start, tip = _centre(300, 200, 23.0, 20.0)
    ps.append(W.with_line_crack(_macro(300, 200), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0))
    start, tip = _centre(300, 200, 61.0, 20.0)
    ps.append(W.with_line_crack(_macro(300, 200), mode="prescribed", start=start, tip=tip, v_rel=0.6, r0=2.0,
                                two_tips=True))
    ps.append(W.with_line_crack(_problem(97, 45), mode="prescribed", start=(10.3, 12.1), tip=(40.6, 30.2), v_rel=0.5))
    return ps


def _same(a, b):
    wa, wda = a.fields()
    wb, wdb = b.fields()
    assert np.array_equal(wa, wb) and np.array_equal(wda, wdb)
    for k in ("h", "v"):
        assert np.array_equal(a.cut_mask(k), b.cut_mask(k))
    assert a.crack_state() == b.crack_state()
    ha, hb = a.history(), b.history()
    for k in ha:
        assert np.array_equal(ha[k], hb[k])


@pytest.mark.parametrize("storage", ["f64", "f32", "f32_bf16"])
@pytest.mark.parametrize("solve", [0, 1])
def test_batch_equals_solo_runs(gpu, storage, solve):
    """One launch per step advances every lattice's line step (tip CTAs and
    march blocks of all lattices), then each lattice with macroscopic faces
    runs its face solve: each lattice ends bit-identical to its solo run."""
    ps = _line_batch_problems()
    solo = [gpu.Lattice(p, storage) for p in ps]
    mem = [gpu.Lattice(p, storage) for p in ps]
    for s_, m in zip(solo, mem):
        s_.set_face_solve(solve)
        m.set_face_solve(solve)
    b = gpu.Batch(mem)
    b.step(1)
    b.step(120)
    for s_ in solo:
        s_.step(121)
    for s_, m in zip(solo, mem):
        _same(s_, m)
    r = b.tune(trial_steps=4)
    assert r["threads"] == 128 and r["lookahead"] == 1
    b.step(30)
    for s_ in solo:
        s_.step(30)
    for s_, m in zip(solo, mem):
        _same(s_, m)
    b.close()


def test_batch_matches_the_oracle(oracle_mod, gpu):
    """The batched lattices against the FP64 oracle: fields within 1e-12,
    both cut masks and the prescribed tips (x and y) exact; the K-criterion
    lattice's tips and K as in test_kcrit_growth_fp64."""
    ps = _line_batch_problems()
    steps = 150
    lats = [gpu.Lattice(p, "f64") for p in ps]
    b = gpu.Batch(lats)
    b.step(steps)
    b.close()
    for p, g in zip(ps, lats):
        o = oracle_mod.Oracle(p)
        o.step(steps)
        _close(o, g, TOL["f64"])
        _masks(o, g)
        ho, hg = _tips(o, g, steps)
        if p["crack"]["mode"] == "kcrit":
            np.testing.assert_allclose(hg["K"], ho["K"], rtol=0, atol=1e-9 * np.abs(ho["K"]).max())
        o.close()
        g.close()


@pytest.mark.parametrize("macro", [False, True])
def test_band_heights_give_the_same_bits(gpu, macro):
    """lbm_set_launch sets the march bands of the step of a crack in any
    direction: every band height gives the same bits (a site's update does
    not depend on which block makes it) through the growth of the crack, and
    0 restores the built-in height."""
    p = W.kcrit_line_centre(scale=8) if macro else W.kcrit_line(scale=8)
    runs = []
    band0 = None
    for rows in (0, 1, 3, 7, 64):
        g = gpu.Lattice(p, "f32")
        if rows == 0:
            band0 = gpu.lbm_get_launch(g.h)["band_rows"]
        else:
            gpu.lbm_set_launch(g.h, rows)
            launch = gpu.lbm_get_launch(g.h)
            assert launch["band_rows"] == rows
            assert launch["ctas"] == 1 + -(-p["nx"] // 512) * -(-p["ny"] // rows)
        g.step(1)
        g.step(600)
        runs.append((g.fields(), g.cut_mask("h"), g.cut_mask("v"), g.crack_state(), g.tip_q()))
        if rows:
            gpu.lbm_set_launch(g.h, 0)
            assert gpu.lbm_get_launch(g.h)["band_rows"] == band0
        g.close()
    (f0, h0, v0, c0, t0) = runs[0]
    for f, h, v, c, t in runs[1:]:
        np.testing.assert_array_equal(f[0], f0[0])
        np.testing.assert_array_equal(f[1], f0[1])
        np.testing.assert_array_equal(h, h0)
        np.testing.assert_array_equal(v, v0)
        assert c == c0 and t == t0
