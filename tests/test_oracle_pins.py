"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

None of these tests compares the oracle with itself: each checks it against a
closed form (dispersion relation of the scheme, synthetic near-tip field,
printed loading formulas), an independently assembled operator (the discrete
Laplacian with the boundary rules, built here from the geometry), an
invariant (energy, momentum, mirror symmetry, static fixed point), brute force
(CheckLinks against every link, exact rational arithmetic), or numbers printed
in the paper (Table 1 of Sec. 5.1).
"""
import math
from fractions import Fraction

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2206_12412_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")

CX = [0, 1, 0, -1, 0]
CY = [0, 0, 1, 0, -1]


# ------------------------------------------------------------- test helpers

def crack_cuts(nx, ny, jc, x_start, x_tip, dh=1.0):
    """Vertical links (i, jc-1)-(i, jc) at x_i = (i + 1/2) dh crossed by the
    closed crack segment [x_start, x_tip] on y = jc dh."""
    cv = np.zeros((ny, nx), bool)
    for i in range(nx):
        if x_start <= (i + 0.5) * dh <= x_tip:
            cv[jc - 1, i] = True
    return cv


def assemble(nx, ny, edges, cut_h, cut_v):
    """Discrete operator of one step written as a graph: for each site p,
    sum over its four links of (value streamed in - w_p) = -(L w)_p + b_p.
    Intact link to q: w_q - w_p.  Severed link or free edge (bounce-back): 0.
    Dirichlet edge (anti-bounce-back): 2 w* - 2 w_p.  Periodic: wrap.
    Returns L (symmetric, csr) and, per edge, the sites with a Dirichlet link."""
    n = nx * ny
    rows, cols, vals = [], [], []
    diag = np.zeros(n)
    dlinks = {e: [] for e in range(4)}

    def idx(i, j):
        return j * nx + i

    for j in range(ny):
        for i in range(nx):
            p = idx(i, j)
            for a, (dx, dy, edge) in enumerate([(1, 0, 1), (-1, 0, 0), (0, 1, 3), (0, -1, 2)]):
                ii, jj = i + dx, j + dy
                outside = not (0 <= ii < nx and 0 <= jj < ny)
                if outside:
                    if edges[edge] == "periodic":
                        ii %= nx
                        jj %= ny
                    elif edges[edge] == "dirichlet":
                        diag[p] += 2.0
                        dlinks[edge].append(p)
                        continue
                    else:
                        continue
                # severed flag of the link
                if dx == 1:
                    cut = cut_h[j, i]
                elif dx == -1:
                    cut = cut_h[jj, ii]
                elif dy == 1:
                    cut = cut_v[j, i]
                else:
                    cut = cut_v[jj, ii]
                if cut:
                    continue
                diag[p] += 1.0
                rows.append(p)
                cols.append(idx(ii, jj))
                vals.append(-1.0)
    L = sp.csr_matrix((vals, (rows, cols)), shape=(n, n)) + sp.diags(diag)
    return L.tocsr(), {e: np.array(v, int) for e, v in dlinks.items()}


def rhs(n, dlinks, wstar):
    b = np.zeros(n)
    for e, sites in dlinks.items():
        np.add.at(b, sites, 2.0 * wstar[e])
    return b


def load_formula(kind, amp, T, t):
    """Printed loading histories: linear ramp; Sec. 5.1 sin^2 ramp; Sec. 5.2 half sine."""
    if kind == "linear":
        return amp if (T <= 0 or t >= T) else amp * t / T
    if kind == "sin2":
        return amp if (T <= 0 or t >= T) else amp * math.sin(math.pi * t / (2 * T)) ** 2
    if kind == "halfsine":
        return 0.0 if t >= T else amp * math.sin(math.pi * t / T)
    if kind == "const":
        return amp
    raise ValueError(kind)


def edge_values(problem, n):
    t = n * problem["dt"]
    ws = [0.0] * 4
    for ld in problem["loads"]:
        e = {"left": 0, "right": 1, "bottom": 2, "top": 3}[ld["edge"]]
        ws[e] = load_formula(ld["kind"], ld["amp"], ld["t"], t)
    return ws


# ------------------------------------------------------ equilibrium moments

def test_equilibrium_moments(oracle_mod):
    """Sec. 3: wdot = sum_a f^a must hold at equilibrium; the first moment
    vanishes and the second is isotropic (2 g w in both directions)."""
    rng = np.random.default_rng(1)
    for _ in range(50):
        w, wd, g = rng.normal(), rng.normal(), rng.uniform(0.01, 0.5)
        f = oracle_mod.equilibrium(w, wd, g)
        assert math.isclose(f.sum(), wd, rel_tol=1e-14, abs_tol=1e-14)
        assert abs(np.dot(CX, f)) < 1e-15 and abs(np.dot(CY, f)) < 1e-15
        assert math.isclose(np.dot(np.square(CX), f), 2 * g * w, rel_tol=1e-14, abs_tol=1e-15)
        assert math.isclose(np.dot(np.square(CY), f), 2 * g * w, rel_tol=1e-14, abs_tol=1e-15)
        assert abs(np.dot(np.multiply(CX, CY), f)) < 1e-15


# --------------------------------------------------------- wave propagation

@pytest.mark.parametrize("m,n", [(1, 0), (3, 2), (5, 7), (24, 16)])
def test_dispersion_relation_periodic(oracle_mod, m, n):
    """A standing mode cos(k.x) on a periodic lattice evolves as
    cos(omega t) with sin^2(omega dt/2) = g dt [sin^2(kx dh/2) + sin^2(ky dh/2)]
    (the scheme is the leapfrog discretisation of the wave equation)."""
    nx, ny = 48, 32
    p = W.base_problem(nx, ny, edges=("periodic",) * 4)
    o = oracle_mod.Oracle(p)
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * n / ny
    X, Y = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    psi = np.cos(kx * X + ky * Y + 0.3)
    gamma = p["mu"] / p["rho"] * p["dt"] ** 2 / p["dh"] ** 2
    om = 2 * math.asin(math.sqrt(gamma * (math.sin(kx / 2) ** 2 + math.sin(ky / 2) ** 2)))
    o.set_fields(psi, (1 - math.cos(om)) / p["dt"] * psi)
    N = 300
    o.step(N)
    w, wd = o.fields()
    assert np.abs(w - math.cos(om * N) * psi).max() < 1e-12
    assert np.abs(wd - (math.cos(om * N) - math.cos(om * (N - 1))) / p["dt"] * psi).max() < 1e-12


@pytest.mark.parametrize("rho,mu", [(1.0, 0.25), (2.0, 0.18), (0.5, 0.06)])
def test_plane_wave_speed(oracle_mod, rho, mu):
    """Long waves travel at c_s = sqrt(mu / rho) (Sec. 2.1).  The angular
    frequency of the projection a_n of w^n on a long plane mode follows from
    a_{n+1} + a_{n-1} = 2 cos(omega dt) a_n, whatever the initial phase."""
    nx, ny = 256, 4
    p = W.base_problem(nx, ny, edges=("periodic",) * 4)
    p["rho"], p["mu"] = rho, mu
    o = oracle_mod.Oracle(p)
    k = 2 * math.pi / nx
    X, _ = np.meshgrid(np.arange(nx) + 0.5, np.arange(ny) + 0.5)
    psi = np.cos(k * X)
    o.set_fields(psi, np.zeros_like(psi))
    a = []
    for _ in range(40):
        o.step(1)
        a.append((o.fields()[0] * psi).sum() / (psi * psi).sum())
    a = np.array(a)
    n = int(np.argmax(np.abs(a[1:-1]))) + 1
    om = math.acos((a[n + 1] + a[n - 1]) / (2 * a[n])) / p["dt"]
    c = math.sqrt(mu / rho)
    assert abs(om / k - c) / c < 1e-3


# ------------------------------------------------- operator and invariants

def _random_problem(bc_mode="bounceback"):
    p = W.base_problem(37, 29, bc_mode=bc_mode, edges=("free", "dirichlet", "dirichlet", "free"))
    p = W.with_crack(p, mode="stationary", y=14.0, x_start=4.3, x_tip=20.7)
    p["loads"] = [{"edge": "right", "kind": "const", "amp": 3e-4, "t": 0.0},
                  {"edge": "bottom", "kind": "sin2", "amp": -5e-4, "t": 40.0}]
    return p


def test_leapfrog_identity_with_boundaries(oracle_mod):
    """w^{n+1} - 2 w^n + w^{n-1} = (c_s dt / dh)^2 (-L w^n + b(w*(t_n))) with the
    operator assembled here from the geometry: bounce-back on free edges and
    crack faces, anti-bounce-back on Dirichlet edges."""
    p = _random_problem()
    nx, ny = p["nx"], p["ny"]
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(nx, ny, seed=11)
    o.set_fields(w0, wd0)
    ch, cv = o.cuts()
    cv_expect = crack_cuts(nx, ny, 14, 4.3, 20.7)
    assert not ch.any() and np.array_equal(cv.astype(bool), cv_expect)
    L, dl = assemble(nx, ny, p["edges"], ch, cv)
    gamma = p["mu"] / p["rho"] * p["dt"] ** 2 / p["dh"] ** 2
    prev = w0.ravel().copy()
    o.step(1)
    cur = o.fields()[0].ravel().copy()
    for n in range(1, 60):
        o.step(1)
        nxt = o.fields()[0].ravel().copy()
        b = rhs(nx * ny, dl, edge_values(p, n))
        resid = (nxt - 2 * cur + prev) - gamma * (-(L @ cur) + b)
        assert np.abs(resid).max() < 1e-14 * max(np.abs(cur).max(), 1e-3), n
        prev, cur = cur, nxt


def test_energy_conserved(oracle_mod):
    """With homogeneous boundary values and a fixed crack, the leapfrog energy
    E = |w^{n+1} - w^n|^2 + gamma (w^{n+1})^T L w^n is conserved."""
    p = W.base_problem(33, 26, bc_mode="bounceback", edges=("free", "dirichlet", "dirichlet", "free"))
    p = W.with_crack(p, mode="stationary", y=13.0, x_tip=15.2)
    nx, ny = p["nx"], p["ny"]
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(nx, ny, seed=5)
    o.set_fields(w0, wd0)
    ch, cv = o.cuts()
    L, _ = assemble(nx, ny, p["edges"], ch, cv)
    gamma = 0.25
    E = []
    prev = w0.ravel().copy()
    for _ in range(400):
        o.step(1)
        cur = o.fields()[0].ravel().copy()
        E.append(np.sum((cur - prev) ** 2) + gamma * cur @ (L @ prev))
        prev = cur
    E = np.array(E)
    assert np.abs(E - E[0]).max() < 1e-12 * abs(E[0])


def test_momentum_conserved_free_edges(oracle_mod):
    """All edges free: sum_x wdot is conserved (the graph Laplacian sums to 0)."""
    p = W.base_problem(31, 22, bc_mode="bounceback", edges=("free",) * 4)
    p = W.with_crack(p, mode="stationary", y=11.0, x_tip=12.0)
    o = oracle_mod.Oracle(p)
    w0, wd0 = W.random_state(31, 22, seed=6)
    o.set_fields(w0, wd0)
    s0 = wd0.sum()
    scale = np.abs(wd0).sum()
    for _ in range(10):
        o.step(25)
        assert abs(o.fields()[1].sum() - s0) < 1e-13 * scale


@pytest.mark.parametrize("bc_mode", ["bounceback", "macroscopic"])
@pytest.mark.parametrize("mode", ["stationary", "prescribed"])
def test_mirror_antisymmetry(oracle_mod, bc_mode, mode):
    """Loading +-u0 antisymmetric about the crack line gives
    w(i, j) = -w(i, ny-1-j) at every step."""
    p = W.base_problem(48, 40, bc_mode=bc_mode)
    p = W.with_crack(p, mode=mode, y=20.0, x_tip=11.3, v_rel=0.35)
    p = W.with_antisymmetric_ramp(p, 1e-3, 30.0)
    o = oracle_mod.Oracle(p)
    for _ in range(8):
        o.step(25)
        w, wd = o.fields()
        assert np.abs(w + w[::-1]).max() < 1e-14 * np.abs(w).max()
        assert np.abs(wd + wd[::-1]).max() < 1e-12 * np.abs(wd).max() + 1e-20


@pytest.mark.parametrize("bc_mode", ["bounceback", "macroscopic"])
def test_static_fixed_point(oracle_mod, bc_mode):
    """The static solution of the discrete problem (solved here with a sparse
    direct solver) is a fixed point of the scheme.  Macroscopic mode: the rows
    of the crack boundary points are replaced by w_B = 1.5 w_I - 0.5 w_II
    (quadratic with zero slope on the face, Sec. 3.1)."""
    nx, ny, jc, tip = 40, 30, 15, 17.6
    p = W.base_problem(nx, ny, bc_mode=bc_mode)
    p = W.with_crack(p, mode="stationary", y=float(jc), x_tip=tip)
    p["loads"] = [{"edge": "top", "kind": "const", "amp": 1e-3, "t": 0.0},
                  {"edge": "bottom", "kind": "const", "amp": -4e-4, "t": 0.0}]
    o = oracle_mod.Oracle(p)
    ch, cv = o.cuts()
    L, dl = assemble(nx, ny, p["edges"], ch, cv)
    b = rhs(nx * ny, dl, edge_values(p, 0))
    A = L.tolil()
    bb = b.copy()
    if bc_mode == "macroscopic":
        for i in np.nonzero(cv[jc - 1])[0]:
            for jB, jI, jII in ((jc - 1, jc - 2, jc - 3), (jc, jc + 1, jc + 2)):
                r = jB * nx + i
                A.rows[r] = []
                A.data[r] = []
                A[r, r] = 1.0
                A[r, jI * nx + i] = -1.5
                A[r, jII * nx + i] = 0.5
                bb[r] = 0.0
    ws = spla.spsolve(A.tocsc(), bb).reshape(ny, nx)
    o.set_fields(ws, np.zeros_like(ws))
    o.step(20)
    w, wd = o.fields()
    assert np.abs(w - ws).max() < 1e-13 * np.abs(ws).max()
    assert np.abs(wd).max() < 1e-15


# ----------------------------------------------------- stress intensity K

@pytest.mark.parametrize("dh", [1.0, 0.5])
@pytest.mark.parametrize("r_min,fit", [(2.0, 1.0), (1.5, 1.0), (2.25, 3.0), (4.0, 6.0)])
def test_K_from_synthetic_near_tip_field(oracle_mod, dh, r_min, fit):
    """Imposing the mode III near-tip field w = (2K/mu) sqrt(r/2pi) sin(phi/2)
    (eq. nearTipDisplacement) with phi = +-pi on the rows next to the crack
    returns K exactly, for one pair (eq. sif) and for a least-squares window."""
    nx, ny, jc = 60, 20, 10
    p = W.base_problem(nx, ny, dh=dh, dt=dh)
    p = W.with_crack(p, mode="stationary", y=jc * dh, x_tip=40.37 * dh)
    o = oracle_mod.Oracle(p)
    mu, K = p["mu"], 0.37
    tip_q = o.crack()["tip_q"]
    w = np.zeros((ny, nx))
    for i in range(nx):
        r = (tip_q / 2**32 - (i + 0.5)) * dh
        if r <= 0:
            continue
        amp = 2 * K / mu * math.sqrt(r / (2 * math.pi))
        w[jc, i], w[jc - 1, i] = amp, -amp
    Kc, npairs = o.evaluate_K(w, tip_q, r_min * dh, fit * dh)
    assert npairs == sum(1 for i in range(nx) if r_min <= tip_q / 2**32 - (i + 0.5) < r_min + fit)
    assert npairs >= 1
    assert abs(Kc - K) < 1e-13 * K


def test_K_single_pair_window(oracle_mod):
    """With W = dh exactly one column is used, the one whose distance r from
    the tip lies in [r_min, r_min + dh); K = delta (mu/4) sqrt(2 pi / r)."""
    nx, ny, jc = 50, 16, 8
    p = W.base_problem(nx, ny)
    p = W.with_crack(p, mode="stationary", y=float(jc), x_tip=30.8)
    o = oracle_mod.Oracle(p)
    tip_q = o.crack()["tip_q"]
    rng = np.random.default_rng(3)
    w = rng.normal(size=(ny, nx))
    for r_min in (0.0, 0.3, 1.0, 2.0, 2.25, 5.5):
        K, npairs = o.evaluate_K(w, tip_q, r_min, 1.0)
        cols = [i for i in range(nx) if r_min <= 30.8 - (i + 0.5) < r_min + 1.0]
        assert npairs == 1 and len(cols) == 1
        i = cols[0]
        r = tip_q / 2**32 - (i + 0.5)
        expect = (w[jc, i] - w[jc - 1, i]) * p["mu"] / 4 * math.sqrt(2 * math.pi / r)
        assert math.isclose(K, expect, rel_tol=1e-14)


def test_K_criterion_velocity_and_advance(oracle_mod):
    """K-criterion runs: v = v_max tanh(sqrt((K/K_C)^4 - 1)) when |K| > K_C
    (eq. v-tanh, evaluated here in 50-digit arithmetic), v = 0 otherwise; the
    tip advances by the nearest 2^-32 dh step to Delta a = v c_s dt."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    p = W.base_problem(96, 48, bc_mode="macroscopic")
    p = W.with_antisymmetric_ramp(p, 2e-3, 100.0)
    K_C = 0.5 * W.strip_reference_K(0.25, 2e-3, 48.0)
    p = W.with_crack(p, mode="kcrit", y=24.0, x_tip=20.0, K_C=K_C, v_max=0.85, r0=2.0)
    o = oracle_mod.Oracle(p)
    o.step(400)
    h = o.history()
    cs = math.sqrt(p["mu"] / p["rho"])
    tip_prev = round(20.0 * 2**32)
    grew = 0
    for n in range(400):
        K, v, np_ = h["K"][n], h["v"][n], h["npairs"][n]
        arrested = tip_prev == p["nx"] * 2**32     # the tip stopped at the far edge
        if np_ > 0 and abs(K) > K_C and not arrested:
            x = mpmath.mpf(abs(K)) / mpmath.mpf(K_C)
            expect = mpmath.mpf(0.85) * mpmath.tanh(mpmath.sqrt(x**4 - 1))
            # rounding of x^4 - 1 in double is amplified by its condition number
            tol = 1e-15 + 8 * 2.2e-16 * float(x**4 / (x**4 - 1))
            assert abs(mpmath.mpf(v) - expect) <= tol * abs(expect)
            grew += 1
        else:
            assert v == 0.0
        step = h["tip_q"][n] - tip_prev
        exact = mpmath.mpf(v) * mpmath.mpf(cs) * p["dt"] / p["dh"] * 2**32
        clamp = p["nx"] * 2**32
        if h["tip_q"][n] == clamp:
            assert tip_prev + exact + 0.5 >= clamp
        else:
            assert abs(step - exact) <= 0.5 + 1e-6
        tip_prev = h["tip_q"][n]
    assert grew > 10   # the run exercises growth


def test_prescribed_advance_cuts_and_clamp(oracle_mod):
    """Prescribed growth: Delta a = v c_s dt per step on the 2^-32 dh grid; the
    severed links are exactly those with x_start <= x_i <= tip (closed
    segment); the tip stops at the far edge x = nx dh, every link of the crack
    row severed."""
    nx, ny, jc = 40, 16, 8
    p = W.base_problem(nx, ny, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=float(jc), x_start=2.5, x_tip=10.0, v_rel=0.6)
    o = oracle_mod.Oracle(p)
    dq = round(0.6 * 0.5 * 2**32)
    tip0 = 10 * 2**32
    for n in range(1, 121):
        o.step(1)
        c = o.crack()
        expect = min(tip0 + n * dq, nx * 2**32)
        assert c["tip_q"] == expect
        _, cv = o.cuts()
        assert np.array_equal(cv.astype(bool), crack_cuts(nx, ny, jc, 2.5, expect / 2**32))
    assert o.crack()["flags"] & 1   # clamped
    bps = set(o.bpoints().tolist())
    cols = np.nonzero(cv[jc - 1])[0]
    assert bps == {jc * nx + i for i in cols} | {(jc - 1) * nx + i for i in cols}


# ------------------------------------------------------------ CheckLinks

def _frac_intersect(p1, p2, q1, q2):
    """Closed segment intersection in exact rational arithmetic (brute force
    via the parametric form, independent of orientation predicates)."""
    (x1, y1), (x2, y2), (x3, y3), (x4, y4) = [tuple(map(Fraction, t)) for t in (p1, p2, q1, q2)]
    d = (x2 - x1) * (y4 - y3) - (y2 - y1) * (x4 - x3)
    if d != 0:
        t = ((x3 - x1) * (y4 - y3) - (y3 - y1) * (x4 - x3)) / d
        u = ((x3 - x1) * (y2 - y1) - (y3 - y1) * (x2 - x1)) / d
        return 0 <= t <= 1 and 0 <= u <= 1
    # parallel (or degenerate): they meet only if one contains an end point of the other
    def on(a, b, c):
        cross = (b[0] - a[0]) * (c[1] - a[1]) - (b[1] - a[1]) * (c[0] - a[0])
        if a == b:
            return c == a
        return cross == 0 and min(a[0], b[0]) <= c[0] <= max(a[0], b[0]) and min(a[1], b[1]) <= c[1] <= max(a[1], b[1])
    P1, P2, Q1, Q2 = (x1, y1), (x2, y2), (x3, y3), (x4, y4)
    return on(P1, P2, Q1) or on(P1, P2, Q2) or on(Q1, Q2, P1) or on(Q1, Q2, P2)


def test_segments_intersect_exact(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(4000):
        pts = [tuple(int(v) for v in rng.integers(-3, 4, size=2)) for _ in range(4)]
        scale = int(rng.choice([1, 2**31, 2**32 + 1]))
        sp_ = [(x * scale, y * scale) for x, y in pts]
        assert oracle_mod.segments_intersect(*sp_) == _frac_intersect(*sp_), sp_


def _brute_links(nx, ny, seg_a, seg_b, cut_h, cut_v):
    """Every intact link of the lattice tested against the segment."""
    found = set()
    for j in range(ny):
        for i in range(nx):
            c = ((2 * i + 1) << 31, (2 * j + 1) << 31)
            if i + 1 < nx and not cut_h[j, i]:
                if _frac_intersect(c, ((2 * i + 3) << 31, c[1]), seg_a, seg_b):
                    found.add(("h", i, j))
            if j + 1 < ny and not cut_v[j, i]:
                if _frac_intersect(c, (c[0], (2 * j + 3) << 31), seg_a, seg_b):
                    found.add(("v", i, j))
    return found


def test_checklinks_matches_brute_force(oracle_mod):
    """Alg. 1 CheckLinks (search from the neighbours of the previous boundary
    points) finds exactly the links a new sub-dh crack segment crosses, for
    random segment directions, on small lattices."""
    rng = np.random.default_rng(8)
    nx = ny = 9
    cases = 0
    for _ in range(600):
        # a previous segment that ends at the old tip, then a new one of length < dh
        a = rng.uniform(2.0, 7.0, size=2)
        ang0 = rng.uniform(0, 2 * np.pi)
        ang1 = ang0 + rng.choice([0.0, rng.uniform(-0.15, 0.15)])   # straight, or a slight kink
        l0, l1 = rng.uniform(0.3, 2.5), rng.uniform(0.05, 0.999)
        s0 = a - l0 * np.array([math.cos(ang0), math.sin(ang0)])
        b = a + l1 * np.array([math.cos(ang1), math.sin(ang1)])
        q = lambda v: (int(round(v[0] * 2**32)), int(round(v[1] * 2**32)))
        S0, A, B = q(s0), q(a), q(b)
        if not all(0 < c < 9 * 2**32 for c in (*S0, *A, *B)):
            continue
        ch = np.zeros((ny, nx), np.uint8)
        cv = np.zeros((ny, nx), np.uint8)
        first = _brute_links(nx, ny, S0, A, ch, cv)
        bprev = set()
        for kind, i, j in first:
            if kind == "h":
                ch[j, i] = 1
                bprev |= {j * nx + i, j * nx + i + 1}
            else:
                cv[j, i] = 1
                bprev |= {j * nx + i, (j + 1) * nx + i}
        expect = _brute_links(nx, ny, A, B, ch, cv)
        got = oracle_mod.checklinks(nx, ny, ch, cv, sorted(bprev), A, B)
        pts = set()
        for kind, i, j in expect:
            pts |= {j * nx + i, j * nx + i + 1} if kind == "h" else {j * nx + i, (j + 1) * nx + i}
            assert (ch if kind == "h" else cv)[j, i] == 1   # severed by CheckLinks
        assert set(got.tolist()) == pts
        cases += 1
    assert cases > 300


# ------------------------------------------------------ macroscopic rule

def test_macroscopic_polynomial(oracle_mod):
    """Quadratic p(s) = a + b s^2 (zero slope on the traction-free face)
    through (s_I, w_I), (s_II, w_II), evaluated at s_B: exact for such
    quadratics, and (3 w_I - w_II)/2 at s = 1/2, 3/2, 5/2."""
    rng = np.random.default_rng(9)
    for _ in range(100):
        a, b = rng.normal(size=2)
        sB = rng.uniform(0.05, 1.0)
        sI, sII = sB + 1.0, sB + 2.0
        got = oracle_mod.macro_poly(sB, sI, sII, a + b * sI**2, a + b * sII**2)
        assert math.isclose(got, a + b * sB**2, rel_tol=1e-12, abs_tol=1e-12)
        wI, wII = rng.normal(size=2)
        assert math.isclose(oracle_mod.macro_poly(0.5, 1.5, 2.5, wI, wII), 1.5 * wI - 0.5 * wII,
                            rel_tol=1e-14, abs_tol=1e-15)
    # a field with non-zero slope at the face is not reproduced (Neumann rule)
    assert abs(oracle_mod.macro_poly(0.5, 1.5, 2.5, 1.5, 2.5) - 0.5) > 0.1


def test_macroscopic_rule_holds_in_run(oracle_mod):
    p = W.plain_fp64("macroscopic")
    o = oracle_mod.Oracle(p)
    o.step(150)
    w, _ = o.fields()
    jc = 64
    for i in range(32):
        assert math.isclose(w[jc, i], 1.5 * w[jc + 1, i] - 0.5 * w[jc + 2, i], rel_tol=1e-13, abs_tol=1e-19)
        assert math.isclose(w[jc - 1, i], 1.5 * w[jc - 2, i] - 0.5 * w[jc - 3, i], rel_tol=1e-13, abs_tol=1e-19)
    assert not math.isclose(w[jc, 40], 1.5 * w[jc + 1, 40] - 0.5 * w[jc + 2, 40], rel_tol=1e-6)


# ---------------------------------------------------------------- loading

def test_loading_histories(oracle_mod):
    """Sec. 5.1 ramp (1/2 w0 sin^2(pi t/(2 t0)), then 1/2 w0), Sec. 5.2 pulse
    (0.01 L sin(pi t / 8) for t < 8, then 0), linear ramp, tabulated series."""
    ser = np.linspace(-1, 1, 17) * 1e-3
    p = W.base_problem(8, 8, edges=("dirichlet",) * 4, dt=0.5, dh=1.0)
    p["loads"] = [{"edge": "left", "kind": "linear", "amp": 2e-3, "t": 50.0},
                  {"edge": "right", "kind": "sin2", "amp": 0.1, "t": 7.0},
                  {"edge": "bottom", "kind": "halfsine", "amp": 0.01, "t": 8.0},
                  {"edge": "top", "kind": "series", "series": ser}]
    o = oracle_mod.Oracle(p)
    for n in (0, 1, 5, 13, 14, 15, 16, 17, 40, 99, 100, 101, 300):
        t = n * 0.5
        assert o.load_value("left", n) == pytest.approx(2e-3 * min(t / 50.0, 1.0), rel=1e-15, abs=0)
        s2 = 0.1 * math.sin(math.pi / 2 * t / 7.0) ** 2 if t < 7.0 else 0.1
        assert o.load_value("right", n) == pytest.approx(s2, rel=1e-15, abs=1e-300)
        hs = 0.01 * math.sin(math.pi * t / 8.0) if t < 8.0 else 0.0
        assert o.load_value("bottom", n) == pytest.approx(hs, rel=1e-15, abs=1e-300)
        assert o.load_value("top", n) == ser[min(n, 16)]


# ------------------------------------------------------- printed numbers

def test_site_counts_cell_centred():
    """Cell-centred sites reproduce the printed lattice sizes (Sec. 5.2: 98304
    points for 8L x 3L at dh = L/64; Sec. 5.3: 10496 points for the v = 0.4
    strip of width 2L at dh = L/16, i.e. 32 rows of 328 sites)."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "paper_counts.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    for wL, hL, dhL, pts in rows:
        nx, ny = round(float(wL) / float(dhL)), round(float(hL) / float(dhL))
        assert nx * ny == int(pts)
        assert (nx + 1) * (ny + 1) != int(pts)
    assert 10496 == 32 * 328 and 2 * 16 == 32


def _table1():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "table1_steady_growth.txt")
    return [tuple(map(float, l.split())) for l in open(path) if l.strip() and not l.startswith("#")]


def test_table1_theory_column_reading():
    """K_theo of Table 1 is eq. sif-mandal with mu = L = 1 and w0 = 0.2."""
    for v, _, Kth, *_ in _table1():
        beta = math.sqrt(1 - v * v)
        assert abs(0.2 * math.sqrt(2 * beta / (2 * beta + 1)) - Kth) < 6e-5


@pytest.mark.parametrize("row", range(4))
def test_table1_steady_growth(oracle_mod, row):
    """Steady growth in a strip of width 2L at dh = L/16 (Sec. 5.1): initial
    crack 0.5 L, edges ramped to +-w0/2 with the sin^2 ramp, crack and sides
    free, the macroscopic rule on the crack faces, r_min from Table 1; the mean
    K over the last 15 L/c_s (300 samples) matches the printed mean within 5 %
    (the paper's domain length and t0 are not printed)."""
    v, rmin, Kth, mean, sigma, *_ = _table1()[row]
    L, u0, t0, tf = 16, 1e-3, 400, 1300
    window = int(15 * L / 0.5)
    nx = 328 if v == 0.4 else int(8 + v * 0.5 * tf + 2 * 2 * L + 8)
    p = W.base_problem(nx, 2 * L, bc_mode="macroscopic")
    p = W.with_crack(p, mode="prescribed", y=float(L), x_tip=0.5 * L, v_rel=v, r_min=rmin)
    p = W.with_antisymmetric_ramp(p, u0, float(t0), kind="sin2")
    o = oracle_mod.Oracle(p)
    o.step(tf)
    K = o.history()["K"][tf - window:]
    K = K[np.linspace(0, window - 1, 300).astype(int)]
    # to Table 1 units: K scales with mu * w0 / sqrt(L); here mu = 1/4, w0 = 2 u0, L = 16 dh
    K_tab = K / (0.25 * 2 * u0 / math.sqrt(L)) * 0.2
    assert abs(K_tab.mean() - mean) < 0.05 * mean, (K_tab.mean(), mean)
