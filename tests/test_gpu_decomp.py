"""Row-slab decomposition (include/lbm_decomp.h): a lattice split into slabs
with halo rows exchanged after every step gives the same bits as the
undivided lattice -- fields, crack state, history and severed links."""
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


def _problem(kind: str):
    if kind == "kcrit_macro":
        p = W.base_problem(300, 96, bc_mode="macroscopic")
        p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
        K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 96.0)
        return W.with_crack(p, mode="kcrit", y=48.0, x_tip=60.0, K_C=K_C, v_max=0.85, r0=2.0)
    if kind == "prescribed_bb":
        p = W.base_problem(530, 77, bc_mode="bounceback", edges=("dirichlet", "free", "dirichlet", "dirichlet"))
        p = W.with_crack(p, mode="prescribed", y=30.0, x_start=4.0, x_tip=100.0, v_rel=0.5)
        rng = np.random.default_rng(3)
        for e in ("left", "bottom", "top"):
            p = W.with_series_load(p, e, 1e-3 * rng.standard_normal(400))
        return p
    if kind == "periodic_y":
        return W.base_problem(129, 64, edges=("free", "dirichlet", "periodic", "periodic"))
    raise KeyError(kind)


def _compare(gpu, p, storage, n_ranks, row_start=None, steps=(7, 64, 100)):
    ref = gpu.Lattice(p, storage)
    dec = gpu.Decomp(p, n_ranks, storage, row_start=row_start)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=n_ranks * 31 + p["ny"],
                             dtype=np.float64 if storage == "f64" else np.float32)
    ref.set_fields(w0, wd0)
    dec.set_fields(w0, wd0)
    for n in steps:
        ref.step(n)
        dec.step(n)
        w_r, wd_r = ref.fields()
        w_d, wd_d = dec.fields()
        np.testing.assert_array_equal(w_d, w_r)
        np.testing.assert_array_equal(wd_d, wd_r)
    info = dec.info()
    if info["crack_rank"] >= 0:
        slab = dec.rank(info["crack_rank"])
        assert slab.crack_state() == ref.crack_state()
        hr, hd = ref.history(), slab.history()
        for k in hr:
            np.testing.assert_array_equal(hd[k], hr[k])
        np.testing.assert_array_equal(slab.cut_mask("v"), ref.cut_mask("v")[slab.row0: slab.row0 + slab.ny])
    dec.close()
    ref.close()
    return info


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("n_ranks", [1, 2, 3, 5])
def test_kcrit_growth_bit_identical(gpu, storage, n_ranks):
    info = _compare(gpu, _problem("kcrit_macro"), storage, n_ranks)
    assert info["n_ranks"] == n_ranks


@pytest.mark.parametrize("row_start", [[0, 2, 77], [0, 27, 33, 77], [0, 29, 31, 40, 75, 77]])
def test_uneven_slabs_with_loaded_edges(gpu, row_start):
    """Bounce-back crack faces (crack rows 29 and 30), slabs ending right at
    the crack rows, two-row slabs, all four edges loaded or free."""
    _compare(gpu, _problem("prescribed_bb"), "f32", len(row_start) - 1, row_start=row_start)


@pytest.mark.parametrize("n_ranks", [2, 4])
def test_periodic_wrap_between_first_and_last_slab(gpu, n_ranks):
    _compare(gpu, _problem("periodic_y"), "f64", n_ranks)


def test_fp16_slabs_share_the_lattice_scale(gpu):
    _compare(gpu, _problem("prescribed_bb"), "f32_f16", 3)


def test_rejects_splits_through_the_crack_rows(gpu):
    p = _problem("kcrit_macro")   # crack rows 45 .. 50 with macroscopic faces, crack line 48
    for rs in ([0, 47, 96], [0, 49, 96], [0, 46, 96], [0, 1, 96], [0, 46, 48, 96]):
        with pytest.raises(gpu.LbmError):
            gpu.Decomp(p, len(rs) - 1, "f32", row_start=rs)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("kind,row_start", [("kcrit_macro", [0, 48, 96]), ("kcrit_macro", [0, 20, 48, 51, 96]),
                                            ("prescribed_bb", [0, 30, 77]), ("prescribed_bb", [0, 12, 30, 32, 77])])
def test_boundary_on_the_crack_line(gpu, storage, kind, row_start):
    """A slab boundary on the crack line: the slabs on both sides hold their
    side's crack rows, read the other side's row from their halo, and each
    runs the crack step -- the same K, decisions and severed links -- so the
    run stays bit-identical to the undivided lattice, and both slabs report
    the undivided lattice's crack state and history."""
    p = _problem(kind)
    info = _compare(gpu, p, storage, len(row_start) - 1, row_start=row_start)
    jc = int(round(p["crack"]["y"]))
    ref = gpu.Lattice(p, storage)
    dec = gpu.Decomp(p, len(row_start) - 1, storage, row_start=row_start)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=5, dtype=np.float64 if storage == "f64" else np.float32)
    ref.set_fields(w0, wd0)
    dec.set_fields(w0, wd0)
    ref.step(150)
    dec.step(150)
    lo, hi = row_start.index(jc) - 1, row_start.index(jc)
    assert info["crack_rank"] == lo
    for r in (lo, hi):
        slab = dec.rank(r)
        assert slab.crack_state() == ref.crack_state()
        hr, hs = ref.history(), slab.history()
        for k in hr:
            np.testing.assert_array_equal(hs[k], hr[k])
    assert (ref.history()["v"] > 0).sum() > 5
    np.testing.assert_array_equal(dec.fields()[0], ref.fields()[0])
    dec.close()
    ref.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_boundary_on_the_crack_line_matches_the_oracle(oracle_mod, gpu, storage):
    from test_gpu_parity import compare_fields
    p = _problem("kcrit_macro")
    dec = gpu.Decomp(p, 2, storage, row_start=[0, 48, 96])
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=17, dtype=np.float64 if storage == "f64" else np.float32)
    dec.set_fields(w0, wd0)
    o.set_fields(w0, wd0)
    dec.step(250)
    o.step(250)
    compare_fields(o, dec, storage)
    ho, hs = o.history(), dec.rank(1).history()
    assert (ho["v"] > 0).sum() > 5
    assert np.abs(hs["K"] - ho["K"]).max() < (1e-9 if storage == "f64" else 5e-3) * np.abs(ho["K"]).max()
    margin = np.min(np.abs(np.abs(ho["K"][ho["npairs"] > 0]) / p["crack"]["K_C"] - 1.0))
    if storage == "f64" and margin > 1e-9:
        np.testing.assert_array_equal(hs["tip_q"], ho["tip_q"])
    o.close()
    dec.close()


# ---------------------------------------------- row slabs vs the oracle

@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("n_ranks", [2, 3, 5])
def test_slabs_match_the_oracle(oracle_mod, gpu, storage, n_ranks):
    """A K-criterion crack with macroscopic faces on a lattice cut into 2, 3
    and 5 row slabs, against the FP64 oracle's undivided run of the same
    problem from the same seeded state: fields within 1e-12 (FP64) / 1e-5
    (FP32) relative max-norm (wdot on the scale of the state), the severed
    links and the tip bit-exact (FP64, where the K decision margin exceeds
    1e-9), K within 1e-9 / 0.5 % of max|K|, the FP32 tip within a spacing."""
    from test_gpu_parity import compare_fields
    p = _problem("kcrit_macro")
    dec = gpu.Decomp(p, n_ranks, storage)
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=n_ranks * 7 + 3,
                             dtype=np.float64 if storage == "f64" else np.float32)
    dec.set_fields(w0, wd0)
    o.set_fields(w0, wd0)
    for n in (1, 99, 200):
        dec.step(n)
        o.step(n)
    compare_fields(o, dec, storage)
    info = dec.info()
    slab = dec.rank(info["crack_rank"])
    co, cs = o.crack(), slab.crack_state()
    ho, hs = o.history(), slab.history()
    assert cs["step"] == co["step"] and len(hs["K"]) == len(ho["K"]) > 0
    assert (ho["v"] > 0).sum() > 5
    K_C = p["crack"]["K_C"]
    kscale = np.abs(ho["K"]).max()
    assert np.abs(hs["K"] - ho["K"]).max() < (1e-9 if storage == "f64" else 5e-3) * kscale
    assert np.array_equal(hs["npairs"], ho["npairs"])
    margin = np.min(np.abs(np.abs(ho["K"][ho["npairs"] > 0]) / K_C - 1.0))
    if storage == "f64" and margin > 1e-9:
        assert cs["tip_q"] == co["tip_q"]
        assert np.array_equal(hs["tip_q"], ho["tip_q"])
        ch, cv = o.cuts()
        np.testing.assert_array_equal(slab.cut_mask("v"), cv.astype(bool)[slab.row0: slab.row0 + slab.ny])
    else:
        assert np.abs(hs["tip_q"] - ho["tip_q"]).max() < 2**32
    o.close()
    dec.close()


# ---------------------------------- the macroscopic rule on every boundary

@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("row_start", [None, [0, 64, 96], [0, 30, 61, 96], [0, 4, 50, 67, 96]])
def test_edge_rule_on_every_boundary_in_slabs(gpu, storage, row_start):
    """The Sec. 5.2 configuration at half size (256 x 96: centre crack, both
    ends growing, the macroscopic rule on every boundary): each slab applies
    the rule to its own edge sites after the step and before the rows are
    exchanged -- the left and right edge points of every slab, the bottom and
    top edges and the corners in the first and last slab, the crack-face
    points on the edge columns in the slabs that hold the crack rows -- so the
    slabs stay bit-identical to the undivided lattice; the boundary may lie on
    the crack line, at the end of the crack rows, or cut a four-row slab."""
    p = W.kcrit_centre_crack(scale=2)
    n_ranks = 3 if row_start is None else len(row_start) - 1
    _compare(gpu, p, storage, n_ranks, row_start=row_start)


def test_edge_rule_slabs_through_crack_growth(gpu):
    """The same problem from rest through the half-sine pulse until both
    ends have grown, on two slabs split at the crack line (both run the
    crack step) and on three."""
    p = W.kcrit_centre_crack(scale=2)
    n = W.KCRIT_CENTRE_STEPS // 2
    ref = gpu.Lattice(p, "f64")
    ref.step(n)
    assert (ref.history(cap=n)["v"] > 0).sum() > 3 and (ref.history_left(cap=n)["v"] > 0).sum() > 3
    w_r, wd_r = ref.fields()
    for rs in ([0, 64, 96], None):
        dec = gpu.Decomp(p, 2 if rs else 3, "f64", row_start=rs)
        dec.step(1)
        dec.step(n - 1)
        w_d, wd_d = dec.fields()
        np.testing.assert_array_equal(w_d, w_r)
        np.testing.assert_array_equal(wd_d, wd_r)
        slab = dec.rank(dec.info()["crack_rank"])
        assert slab.crack_state() == ref.crack_state()
        np.testing.assert_array_equal(slab.history(cap=n)["tip_q"], ref.history(cap=n)["tip_q"])
        np.testing.assert_array_equal(slab.history_left(cap=n)["tip_q"], ref.history_left(cap=n)["tip_q"])
        dec.close()
    ref.close()


def test_edge_rule_slabs_match_the_oracle(oracle_mod, gpu):
    """Three slabs with the macroscopic rule on every boundary against the
    FP64 oracle's undivided run: fields within 1e-12 of max(max|w|, 2 max|w*|)
    (the Dirichlet values dominate the scale), the cut mask and both tips
    exact."""
    p = W.kcrit_centre_crack(scale=2)
    n = 800
    dec = gpu.Decomp(p, 3, "f64")
    o = oracle_mod.Oracle(p)
    dec.step(n)
    o.step(n)
    wo, wdo = o.fields()
    wg, wdg = dec.fields()
    ws = max(abs(L.get("amp", 0.0)) for L in p["loads"])
    scale = max(np.abs(wo).max(), 2 * ws)
    assert np.abs(wg - wo).max() <= 1e-12 * scale and np.abs(wdg - wdo).max() <= 1e-12 * scale
    slab = dec.rank(dec.info()["crack_rank"])
    np.testing.assert_array_equal(slab.history(cap=n)["tip_q"], o.history()["tip_q"][:n])
    np.testing.assert_array_equal(slab.history_left(cap=n)["tip_q"], o.history_left()["tip_q"][:n])
    ch, cv = o.cuts()
    np.testing.assert_array_equal(slab.cut_mask("v"), cv.astype(bool)[slab.row0: slab.row0 + slab.ny])
    o.close()
    dec.close()


def test_edge_rule_slab_handles_exchanging_on_the_host(gpu):
    """One slab handle per part (the per-process form, lbm_slab_*), boundary
    rows exported and imported on the host after every step: with the
    macroscopic rule on every boundary, bit-identical to the undivided
    lattice."""
    p = W.kcrit_centre_crack(scale=2)
    rs = [0, 40, 64, 96]
    ref = gpu.Lattice(p, "f32")
    slabs = [gpu.Slab(p, rs[r], rs[r + 1] - rs[r], "f32") for r in range(3)]

    def exchange():
        rows = [s.export_rows() for s in slabs]
        for r, s in enumerate(slabs):
            s.import_rows(rows[r - 1][1] if r > 0 else None, rows[r + 1][0] if r < 2 else None)

    exchange()
    for _ in range(150):
        for s in slabs:
            s.step(1)
        exchange()
    ref.step(150)
    w_r, wd_r = ref.fields()
    for r, s in enumerate(slabs):
        w, wd = s.fields()
        np.testing.assert_array_equal(w, w_r[rs[r]: rs[r + 1]])
        np.testing.assert_array_equal(wd, wd_r[rs[r]: rs[r + 1]])
        s.close()
    ref.close()
