"""D2Q9 lattices (LBM_D2Q9) in row slabs (include/lbm_decomp.h): the
nine-point update reads rows j-1, j, j+1 only, so one halo row per side
carries every neighbour, diagonals included.  A split keeps the crack rows in
one slab (no boundary on the crack line for D2Q9).  Slabs give the same bits
as the undivided D2Q9 lattice -- fields, crack state, history and severed
links -- on one device (lbm_decomp_*) and as slab handles exchanging their
boundary rows on the host (lbm_slab_*), and stay within parity of the FP64
oracle's undivided D2Q9 run."""
import numpy as np
import pytest

from paper_2206_12412_gb300 import workloads as W
from test_gpu_decomp import _compare

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2206_12412_gb300 import lbm
    lbm.load_library()
    return lbm


def _d2q9(kind: str) -> dict:
    if kind == "kcrit_macro":
        # crack rows 45 .. 50 (macroscopic faces), crack line 48
        p = W.base_problem(300, 96, bc_mode="macroscopic")
        p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
        K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 96.0)
        p = W.with_crack(p, mode="kcrit", y=48.0, x_tip=60.0, K_C=K_C, v_max=0.85, r0=2.0)
    elif kind == "prescribed_bb":
        # crack rows 29 and 30 (bounce-back faces), every edge loaded or free
        p = W.base_problem(530, 77, bc_mode="bounceback", edges=("dirichlet", "free", "dirichlet", "dirichlet"))
        p = W.with_crack(p, mode="prescribed", y=30.0, x_start=4.0, x_tip=100.0, v_rel=0.5)
        rng = np.random.default_rng(3)
        for e in ("left", "bottom", "top"):
            p = W.with_series_load(p, e, 1e-3 * rng.standard_normal(400))
    elif kind == "periodic_y":
        p = W.base_problem(129, 64, edges=("free", "dirichlet", "periodic", "periodic"))
    elif kind == "centre_edges":
        # the Sec. 5.2 configuration at half size: 256 x 96, crack line 64
        # (rows 61 .. 66), both ends growing, the macroscopic rule on every
        # boundary
        p = W.kcrit_centre_crack(scale=2)
    else:
        raise KeyError(kind)
    p["lattice"] = "D2Q9"
    return p


def _f32_tol(n: int, g: float = 0.25) -> float:
    # the leapfrog is neutral, so FP32 rounding accumulates: each step rounds
    # w and a sum of terms up to (16 g / 3) max|w| (the bound the single D2Q9
    # lattice's tests use)
    return max(1e-5, 2 * n * (1 + 16 * g / 3) * 2.0 ** -24)


@pytest.mark.parametrize("storage", ["f32", "f64"])
@pytest.mark.parametrize("n_ranks", [2, 3, 5])
def test_kcrit_growth_bit_identical(gpu, storage, n_ranks):
    """K-criterion growth with macroscopic crack faces: the planned split
    moves a boundary that falls in the crack rows to their nearer end, never
    onto the crack line."""
    info = _compare(gpu, _d2q9("kcrit_macro"), storage, n_ranks)
    assert info["n_ranks"] == n_ranks and info["crack_rank"] >= 0


@pytest.mark.parametrize("row_start", [[0, 29, 31, 77], [0, 2, 29, 31, 40, 75, 77], [0, 31, 77]])
def test_uneven_slabs_with_loaded_edges(gpu, row_start):
    """Bounce-back crack faces on rows 29 and 30: a two-row slab holding just
    the crack rows, slabs ending right at them, two-row slabs at the edges,
    all four edges loaded or free (the diagonal links leaving a corner)."""
    _compare(gpu, _d2q9("prescribed_bb"), "f32", len(row_start) - 1, row_start=row_start)


@pytest.mark.parametrize("n_ranks", [2, 4])
def test_periodic_wrap_between_first_and_last_slab(gpu, n_ranks):
    _compare(gpu, _d2q9("periodic_y"), "f64", n_ranks)


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("row_start", [None, [0, 30, 61, 96], [0, 4, 50, 67, 96]])
def test_edge_rule_on_every_boundary_in_slabs(gpu, storage, row_start):
    """The macroscopic rule on every boundary of a D2Q9 lattice: each slab
    applies it to its own edge sites after its step and before the exchange
    (a corner's diagonal links need no other slab's sites), so the slabs stay
    bit-identical to the undivided lattice."""
    p = _d2q9("centre_edges")
    n_ranks = 3 if row_start is None else len(row_start) - 1
    _compare(gpu, p, storage, n_ranks, row_start=row_start)


def test_rejects_boundaries_in_the_crack_rows(gpu):
    """A D2Q9 boundary may not lie in the crack rows, the crack line
    included (D2Q5 allows the line)."""
    p = _d2q9("centre_edges")   # crack line 64, crack rows 61 .. 66
    for rs in ([0, 64, 96], [0, 62, 96], [0, 66, 96], [0, 30, 64, 96]):
        with pytest.raises(gpu.LbmError):
            gpu.Decomp(p, len(rs) - 1, "f32", row_start=rs)
    for row0, rows in ((0, 64), (64, 32), (0, 63)):
        with pytest.raises(gpu.LbmError):
            gpu.Slab(p, row0, rows, "f32")


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_slabs_match_the_oracle(oracle_mod, gpu, storage):
    """Three D2Q9 slabs with a K-criterion crack and macroscopic faces
    against the FP64 oracle's undivided D2Q9 run from the same seeded state:
    fields within 1e-12 (FP64) or the FP32 accumulation bound, K within 1e-9
    (FP64) / 0.5 % (FP32) of max|K|, the pair counts exact, the severed links
    and tip exact in FP64 where the K decision margin exceeds 1e-9."""
    p = _d2q9("kcrit_macro")
    n = 300
    dec = gpu.Decomp(p, 3, storage)
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(p["nx"], p["ny"], seed=41, dtype=np.float64 if storage == "f64" else np.float32)
    dec.set_fields(w0, wd0)
    o.set_fields(w0, wd0)
    for k in (1, 99, 200):
        dec.step(k)
        o.step(k)
    wo, wdo = o.fields()
    wg, wdg = dec.fields()
    scale = np.abs(wo).max()
    tol = 1e-12 if storage == "f64" else _f32_tol(n)
    assert np.abs(wg - wo).max() <= tol * scale
    assert np.abs(wdg - wdo).max() <= tol * scale
    slab = dec.rank(dec.info()["crack_rank"])
    ho, hs = o.history(), slab.history()
    assert len(hs["K"]) == len(ho["K"]) > 0 and (ho["v"] > 0).sum() > 5
    assert np.abs(hs["K"] - ho["K"]).max() < (1e-9 if storage == "f64" else 5e-3) * np.abs(ho["K"]).max()
    assert np.array_equal(hs["npairs"], ho["npairs"])
    margin = np.min(np.abs(np.abs(ho["K"][ho["npairs"] > 0]) / p["crack"]["K_C"] - 1.0))
    if storage == "f64" and margin > 1e-9:
        np.testing.assert_array_equal(hs["tip_q"], ho["tip_q"])
        np.testing.assert_array_equal(slab.cut_mask("v"), o.cuts()[1].astype(bool)[slab.row0: slab.row0 + slab.ny])
    else:
        assert np.abs(hs["tip_q"] - ho["tip_q"]).max() < 2 ** 32
    o.close()
    dec.close()


def test_edge_rule_slabs_match_the_oracle(oracle_mod, gpu):
    """Three D2Q9 slabs with the macroscopic rule on every boundary, from
    rest through the pulse, against the FP64 oracle's undivided D2Q9 run:
    every growth decision and cut link as the oracle's, both tips within 2
    units of the 2^-32 dh grid (K summed in another order differs in its last
    bits; near K_C eq. v-tanh magnifies that by one unit at most), fields
    within max(1e-12, 2 n (1 + 16 g / 3) 2^-53) of max(max|w|, 2 max|w*|)."""
    p = _d2q9("centre_edges")
    n = 800
    dec = gpu.Decomp(p, 3, "f64")
    o = oracle_mod.Oracle(p)
    dec.step(n)
    o.step(n)
    slab = dec.rank(dec.info()["crack_rank"])
    for hs, ho in ((slab.history(cap=n), o.history()), (slab.history_left(cap=n), o.history_left())):
        np.testing.assert_array_equal(hs["v"] > 0, ho["v"][:n] > 0)
        assert np.abs(hs["tip_q"] - ho["tip_q"][:n]).max() <= 2
    np.testing.assert_array_equal(slab.cut_mask("v"), o.cuts()[1].astype(bool)[slab.row0: slab.row0 + slab.ny])
    wo, wdo = o.fields()
    wg, wdg = dec.fields()
    ws = max(abs(L.get("amp", 0.0)) for L in p["loads"])
    scale = max(np.abs(wo).max(), 2 * ws)
    tol = max(1e-12, 2 * n * (1 + 16 * 0.25 / 3) * 2.0 ** -53)
    assert np.abs(wg - wo).max() <= tol * scale and np.abs(wdg - wdo).max() <= tol * scale
    o.close()
    dec.close()


def test_slab_handles_exchanging_on_the_host(gpu):
    """One D2Q9 slab handle per part (the per-process form), boundary rows
    exported and imported on the host after every step, the macroscopic rule
    on every boundary: bit-identical to the undivided lattice."""
    p = _d2q9("centre_edges")
    rs = [0, 40, 67, 96]
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
