"""Seeded synthetic workloads shaped like the paper's problems.

Problem dicts only (lattice, material, edges, crack, loads) and seeded random
inputs; nothing here computes any part of the method.  Both the CUDA binding
(``lbm.Lattice``) and the CPU oracle read these dicts, so that both sides are
always given the same inputs.

Lattice units throughout: dh = dt = 1, rho = 1, c_s = 0.5 (mu = 0.25), which
gives c = dh/dt = 2 c_s (kappa = 2 in Sec. 4.1) and g = c_s^2 dt^2/dh^2 = 1/4.
"""
from __future__ import annotations

import math

import numpy as np

DEFAULT_HIST_CAP = 1 << 16


def base_problem(nx: int, ny: int, *, bc_mode: str = "macroscopic", edges=("free", "free", "dirichlet", "dirichlet"),
                 cs: float = 0.5, rho: float = 1.0, dh: float = 1.0, dt: float = 1.0) -> dict:
    return {
        "nx": int(nx), "ny": int(ny), "dh": float(dh), "dt": float(dt),
        "edges": tuple(edges), "rho": float(rho), "mu": float(rho * cs * cs), "omega": 1.0,
        "bc_mode": bc_mode, "crack": {"mode": "none"}, "loads": [], "hist_cap": DEFAULT_HIST_CAP,
    }


def with_crack(p: dict, *, mode: str, y: float, x_tip: float, x_start: float = 0.0, v_rel: float = 0.0,
               K_C: float = 0.0, v_max: float = 0.85, r0: float = 2.0, r_min: float = 0.0,
               fit_width: float = 1.0, two_tips: bool = False) -> dict:
    """A straight crack on y from x_start to x_tip; with two_tips the end at
    x_start grows too (towards -x)."""
    q = dict(p)
    q["crack"] = {"mode": mode, "y": float(y), "x_start": float(x_start), "x_tip": float(x_tip),
                  "v_rel": float(v_rel), "K_C": float(K_C), "v_max": float(v_max), "r0": float(r0),
                  "r_min": float(r_min), "fit_width": float(fit_width), "two_tips": bool(two_tips)}
    return q


def with_line_crack(p: dict, *, mode: str, start, tip, v_rel: float = 0.0, K_C: float = 0.0, v_max: float = 0.85,
                    r0: float = 2.0, r_min: float = 0.0, fit_width: float = 1.0, two_tips: bool = False) -> dict:
    """A straight crack in any direction (Sec. 4.1): from start = (x, y)
    through tip = (x, y), growing from the tip along that direction; with
    two_tips the start grows too, the opposite way."""
    q = dict(p)
    q["crack"] = {"mode": mode, "x_start": float(start[0]), "y_start": float(start[1]), "x_tip": float(tip[0]),
                  "y_tip": float(tip[1]), "v_rel": float(v_rel), "K_C": float(K_C), "v_max": float(v_max),
                  "r0": float(r0), "r_min": float(r_min), "fit_width": float(fit_width), "two_tips": bool(two_tips)}
    return q


def with_antisymmetric_ramp(p: dict, u0: float, t_ramp: float, kind: str = "linear") -> dict:
    """Top edge +u0, bottom edge -u0, ramped over t_ramp."""
    q = dict(p)
    q["loads"] = [{"edge": "top", "kind": kind, "amp": float(u0), "t": float(t_ramp)},
                  {"edge": "bottom", "kind": kind, "amp": -float(u0), "t": float(t_ramp)}]
    return q


def strip_reference_K(mu: float, u0: float, height: float) -> float:
    """Textbook LEFM value for a semi-infinite crack on the midline of a strip
    of the given height whose edges are held at +-u0: K0 = mu * 2 u0 /
    sqrt(height).  Used only to pick a critical K_C of the right magnitude."""
    return mu * 2.0 * u0 / math.sqrt(height)


# ------------------------------------------------------------------ configs

def plain_fp64(bc_mode: str = "macroscopic") -> dict:
    """128x128, crack on y = 64 from x = 0 to 32, stationary, +-1e-3 on the
    top/bottom edges ramped linearly over 200 steps; run for 2000 steps."""
    p = base_problem(128, 128, bc_mode=bc_mode)
    p = with_crack(p, mode="stationary", y=64.0, x_tip=32.0, r0=2.0)
    return with_antisymmetric_ramp(p, 1e-3, 200.0)


PLAIN_FP64_STEPS = 2000


def kcrit_single(scale: int = 1, seed: int = 2, bc_mode: str = "macroscopic") -> dict:
    """4096x2048 / scale: edge crack to x = 512 / scale on the midline, top and
    bottom ramped to +-2e-3 over 5000 / scale steps, K-criterion with
    v_max = 0.85, r0 = 2 dh and K_C = 0.5 K_ref (1 + 0.1 U(-1, 1)) drawn from
    the seed, so that growth starts around mid-ramp."""
    nx, ny = 4096 // scale, 2048 // scale
    rng = np.random.default_rng(seed)
    K_ref = strip_reference_K(0.25, 2e-3, float(ny))
    K_C = 0.5 * K_ref * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    p = base_problem(nx, ny, bc_mode=bc_mode)
    p = with_crack(p, mode="kcrit", y=float(ny // 2), x_tip=512.0 / scale, K_C=K_C, v_max=0.85, r0=2.0)
    return with_antisymmetric_ramp(p, 2e-3, 5000.0 / scale)


KCRIT_SINGLE_STEPS = 50000


def large_prescribed(n: int = 16384, bc_mode: str = "macroscopic") -> dict:
    """n x n (16384 x 16384: 268 M sites, 4.3 GB of FP32 state): an edge crack
    on the midline from 0 to n / 8 growing at the prescribed v = 0.5 c_s,
    top and bottom ramped to +-1e-3 over 2000 steps; 20 000 steps (it advances
    0.25 dh per step, so at n = 16384 the tip goes from 2048 to 7048)."""
    p = base_problem(n, n, bc_mode=bc_mode)
    p = with_crack(p, mode="prescribed", y=float(n // 2), x_tip=n / 8.0, v_rel=0.5)
    p = with_antisymmetric_ramp(p, 1e-3, 2000.0)
    p["hist_cap"] = 4096
    return p


LARGE_PRESCRIBED_STEPS = 20000


def kcrit_line(scale: int = 1, seed: int = 2, degrees: float = 20.0) -> dict:
    """kcrit_single with the crack in another direction (Sec. 4.1): an edge
    crack from (0, ny/2 - 0.3) of length 512 / scale at `degrees` to +x,
    link-local faces, the same loads and K-criterion; K_C is 0.35 K_ref
    (1 + 0.1 U(-1, 1)), so that the inclined crack, loaded partly across its
    faces, starts growing around mid-ramp too."""
    nx, ny = 4096 // scale, 2048 // scale
    rng = np.random.default_rng(seed)
    K_C = 0.35 * strip_reference_K(0.25, 2e-3, float(ny)) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    th = math.radians(degrees)
    start = (0.0, ny / 2 - 0.3)
    tip = (start[0] + 512.0 / scale * math.cos(th), start[1] + 512.0 / scale * math.sin(th))
    p = base_problem(nx, ny, bc_mode="bounceback")
    p = with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, v_max=0.85, r0=2.0)
    return with_antisymmetric_ramp(p, 2e-3, 5000.0 / scale)


def kcrit_line_centre(scale: int = 1, seed: int = 2, degrees: float = 20.0, bc_mode: str = "macroscopic") -> dict:
    """kcrit_line with a centre crack instead: length 512 / scale at `degrees`
    to +x through the middle of the body (offset by a small fraction of a
    spacing, so that its line meets no site centre), both ends growing, the
    macroscopic rule on its faces by default (its stencils stay inside the
    body, which an edge crack's would not at the mouth)."""
    nx, ny = 4096 // scale, 2048 // scale
    rng = np.random.default_rng(seed)
    K_C = 0.35 * strip_reference_K(0.25, 2e-3, float(ny)) * (1.0 + 0.1 * rng.uniform(-1.0, 1.0))
    th = math.radians(degrees)
    half = 256.0 / scale
    mid = (nx / 2 + 0.013, ny / 2 + 0.007)
    start = (mid[0] - half * math.cos(th), mid[1] - half * math.sin(th))
    tip = (mid[0] + half * math.cos(th), mid[1] + half * math.sin(th))
    p = base_problem(nx, ny, bc_mode=bc_mode)
    p = with_line_crack(p, mode="kcrit", start=start, tip=tip, K_C=K_C, v_max=0.85, r0=2.0, two_tips=True)
    return with_antisymmetric_ramp(p, 2e-3, 5000.0 / scale)


def kcrit_centre_crack(scale: int = 1, bc_mode: str = "macroscopic_edges") -> dict:
    """The K-criterion example of Sec. 5.2 with L = 64 / scale dh: an 8L x 3L
    body (512 x 192 sites at scale 1), a centre crack of length L on the line
    2L above the bottom edge (x in [3.5L, 4.5L]) whose two tips both grow,
    K_C = 0.0055 mu sqrt(L), r0 = 0.03 L (about 2 dh at scale 1, kept at 2 dh),
    v_max = 0.85; the bottom edge held at w* = 0, the top edge driven by
    0.01 L sin(pi t / (8 L / c_s)) for t < 8 L / c_s and 0 afterwards, the
    lateral edges and the crack faces traction free; the macroscopic rule on
    every boundary.  Runs KCRIT_CENTRE_STEPS / scale steps (39.5 L / c_s)."""
    Lh = 64 // scale
    cs = 0.5
    p = base_problem(8 * Lh, 3 * Lh, bc_mode=bc_mode, edges=("free", "free", "dirichlet", "dirichlet"), cs=cs)
    mu = p["mu"]
    p = with_crack(p, mode="kcrit", y=float(2 * Lh), x_start=3.5 * Lh, x_tip=4.5 * Lh,
                   K_C=0.0055 * mu * math.sqrt(Lh), v_max=0.85, r0=2.0, two_tips=True)
    p["loads"] = [{"edge": "bottom", "kind": "zero"},
                  {"edge": "top", "kind": "halfsine", "amp": 0.01 * Lh, "t": 8.0 * Lh / cs}]
    return p


KCRIT_CENTRE_STEPS = 5050


def prescribed_strip(nx: int, ny: int, v_rel: float, *, u0: float = 1e-3, t_ramp: float = 200.0,
                     crack_len: float | None = None, r_min: float = 0.0, bc_mode: str = "macroscopic") -> dict:
    """Strip with a midline edge crack growing at the prescribed speed."""
    p = base_problem(nx, ny, bc_mode=bc_mode)
    p = with_crack(p, mode="prescribed", y=float(ny // 2), x_tip=crack_len if crack_len is not None else nx / 4,
                   v_rel=v_rel, r_min=r_min)
    return with_antisymmetric_ramp(p, u0, t_ramp)


# ------------------------------------------------------------ random inputs

def smooth_field(nx: int, ny: int, seed: int, amp: float = 1e-3, modes: int = 6) -> np.ndarray:
    """Sum of a few random Fourier modes plus small white noise, (ny, nx) FP64."""
    rng = np.random.default_rng(seed)
    x = (np.arange(nx) + 0.5) / nx
    y = (np.arange(ny) + 0.5) / ny
    X, Y = np.meshgrid(x, y)
    f = np.zeros((ny, nx))
    for _ in range(modes):
        kx, ky = rng.integers(1, 6, size=2)
        ph = rng.uniform(0, 2 * np.pi, size=2)
        f += rng.normal() * np.sin(2 * np.pi * kx * X + ph[0]) * np.cos(2 * np.pi * ky * Y + ph[1])
    f += 0.05 * rng.standard_normal((ny, nx))
    return amp * f / max(np.abs(f).max(), 1e-300)


def random_state(nx: int, ny: int, seed: int, amp: float = 1e-3, dtype=np.float64):
    """Seeded (w, wdot) pair; rounded to `dtype` first so that both sides start
    from bit-identical values."""
    w = smooth_field(nx, ny, seed, amp)
    wd = smooth_field(nx, ny, seed + 7919, amp * 0.05)
    return w.astype(dtype).astype(np.float64), wd.astype(dtype).astype(np.float64)


def batch_problems(n: int = 256, seed: int = 3, bc_mode: str = "macroscopic") -> list:
    """Independent fracture runs of uneven sizes: nx in {256, 288, ..., 1024},
    ny in {128, 160, ..., 512}, an edge crack of U(0.1, 0.4) nx on the
    midline, top/bottom +-u0 with u0 log-uniform in [5e-4, 5e-3] ramped over
    1000 steps; half of them grow by the K-criterion with K_C = K_ref
    U(0.7, 1.3), half at a prescribed v / c_s ~ U(0.1, 0.7)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        nx = int(rng.integers(256 // 32, 1024 // 32 + 1)) * 32
        ny = int(rng.integers(128 // 32, 512 // 32 + 1)) * 32
        length = float(rng.uniform(0.1, 0.4)) * nx
        u0 = float(np.exp(rng.uniform(np.log(5e-4), np.log(5e-3))))
        p = base_problem(nx, ny, bc_mode=bc_mode)
        if rng.uniform() < 0.5:
            K_C = strip_reference_K(0.25, u0, float(ny)) * float(rng.uniform(0.7, 1.3))
            p = with_crack(p, mode="kcrit", y=float(ny // 2), x_tip=length, K_C=K_C, v_max=0.85, r0=2.0)
        else:
            p = with_crack(p, mode="prescribed", y=float(ny // 2), x_tip=length, v_rel=float(rng.uniform(0.1, 0.7)))
        p = with_antisymmetric_ramp(p, u0, 1000.0)
        p["hist_cap"] = 4096
        out.append(p)
    return out


BATCH_STEPS = 20000


# ------------------------------------------------------------------ adjoint

def gp_series(n: int, length: float, sigma: float, seed: int) -> np.ndarray:
    """Smooth random series of n samples: white noise filtered in the
    frequency domain by the square root of a squared-exponential spectrum of
    correlation length `length` (samples), scaled to standard deviation
    sigma over a draw of at least 8 correlation lengths (of which the first n
    samples are returned).  FP64."""
    rng = np.random.default_rng(seed)
    m = max(int(n), int(np.ceil(8 * length)))   # at least 8 correlation lengths, so the scale is well defined
    z = rng.standard_normal(m)
    f = np.fft.rfftfreq(m)
    filt = np.exp(-(np.pi * length * f) ** 2)   # sqrt of exp(-2 pi^2 l^2 f^2)
    x = np.fft.irfft(np.fft.rfft(z) * filt, m)
    return (sigma * x / max(float(np.std(x)), 1e-300))[: int(n)]


def sensor_sites(nx: int, ny: int, ns: int, seed: int, jc: int | None = None, margin: int = 2) -> np.ndarray:
    """ns distinct sites (i, j) drawn uniformly, keeping `margin` rows and
    columns away from the edges and `margin` rows away from the crack rows
    jc-1 and jc.  (ns, 2) int32."""
    rng = np.random.default_rng(seed)
    out, seen = [], set()
    while len(out) < ns:
        i = int(rng.integers(margin, nx - margin))
        j = int(rng.integers(margin, ny - margin))
        if jc is not None and jc - 1 - margin <= j <= jc + margin:
            continue
        if (i, j) in seen:
            continue
        seen.add((i, j))
        out.append((i, j))
    return np.asarray(out, dtype=np.int32)


def with_series_load(p: dict, edge: str, series) -> dict:
    """Replace (or add) the load of one Dirichlet edge by a tabulated series
    (value series[n] in step n)."""
    q = dict(p)
    q["loads"] = [ld for ld in p.get("loads", []) if ld["edge"] != edge]
    q["loads"].append({"edge": edge, "kind": "series", "series": np.asarray(series, dtype=np.float64)})
    return q


def adjoint_problem(nx: int = 1024, ny: int = 1024, n_steps: int = 8000, ns: int = 64, *, crack_len: float | None = None,
                    v_rel: float = 0.4, length: float = 500.0, sigma: float = 1e-3, bc_mode: str = "macroscopic",
                    seeds=(4, 5, 6)) -> dict:
    """Sensor-misfit problem on an nx x ny strip (1024 x 1024, 8000 steps,
    64 sensors at full size): crack on the midline from x = 0 to nx / 8
    growing at the prescribed v / c_s = v_rel; top edge held at a series u[n],
    bottom edge at 0, sides free.  Returns the problem for the control series
    (seed seeds[2]), the reference series whose sensor trace gives the
    targets (seed seeds[0]), and the sensor sites (seed seeds[1])."""
    jc = ny // 2
    p = base_problem(nx, ny, bc_mode=bc_mode)
    p = with_crack(p, mode="prescribed", y=float(jc), x_tip=crack_len if crack_len is not None else nx / 8.0, v_rel=v_rel)
    u_ref = gp_series(n_steps, length, sigma, seeds[0])
    u_ctl = gp_series(n_steps, length, sigma, seeds[2])
    p = with_series_load(p, "top", u_ctl)
    p["hist_cap"] = 4096
    sens = sensor_sites(nx, ny, ns, seeds[1], jc=jc)
    return {"problem": p, "u_ref": u_ref, "u_ctl": u_ctl, "sensors": sens, "n_steps": int(n_steps)}


ADJOINT_STEPS = 8000


def adjoint_case(kind: str, n_steps: int, seed: int, ns: int = 6):
    """Small sensor-misfit problems whose cut schedule does not depend on the
    fields (stationary or prescribed cracks), each Dirichlet edge loaded by a
    seeded random series, with random initial fields, sensors and targets.
    Returns (problem, loaded edges, w0, wd0, sensors (ns, 2), targets
    (n_steps, ns)).  The "wide_*" kinds span several column blocks of the
    CUDA kernels with a ragged last block."""
    rng = np.random.default_rng(seed)
    T = int(n_steps)
    if kind == "macro_growth":
        p = base_problem(24, 20, bc_mode="macroscopic")
        p = with_crack(p, mode="prescribed", y=10.0, x_tip=5.3, v_rel=0.6)
        loaded = ("bottom", "top")
    elif kind == "bb_growth":
        p = base_problem(22, 18, bc_mode="bounceback")
        p = with_crack(p, mode="prescribed", y=9.0, x_tip=4.0, v_rel=0.5)
        loaded = ("bottom", "top")
    elif kind == "bb_periodic":
        p = base_problem(20, 16, bc_mode="bounceback", edges=("periodic", "periodic", "dirichlet", "free"))
        p = with_crack(p, mode="stationary", y=8.0, x_start=3.0, x_tip=11.0)
        loaded = ("bottom",)
    elif kind == "all_dirichlet":
        p = base_problem(18, 15, bc_mode="macroscopic", edges=("dirichlet", "free", "dirichlet", "dirichlet"))
        p = with_crack(p, mode="prescribed", y=7.0, x_start=6.0, x_tip=8.0, v_rel=0.3)
        loaded = ("left", "bottom", "top")
    elif kind == "scaled_units":
        # dh, dt and c_s away from 1, so that every factor of dt, dh and g shows
        p = base_problem(20, 18, bc_mode="macroscopic", cs=0.7, dh=0.5, dt=0.3)
        p = with_crack(p, mode="prescribed", y=4.5, x_tip=2.6, v_rel=0.5)
        loaded = ("bottom", "top")
    elif kind == "no_crack":
        p = base_problem(16, 14, edges=("free", "dirichlet", "periodic", "periodic"))
        loaded = ("right",)
    elif kind == "wide_macro":
        p = base_problem(1100, 70, bc_mode="macroscopic", edges=("dirichlet", "free", "dirichlet", "dirichlet"))
        p = with_crack(p, mode="prescribed", y=37.0, x_tip=500.7, v_rel=0.7)
        loaded = ("left", "bottom", "top")
    elif kind == "wide_bb":
        p = base_problem(777, 41, bc_mode="bounceback", edges=("free", "dirichlet", "dirichlet", "free"))
        p = with_crack(p, mode="prescribed", y=20.0, x_start=3.0, x_tip=505.0, v_rel=0.4)
        loaded = ("right", "bottom")
    else:
        raise KeyError(kind)
    for e in loaded:
        p = with_series_load(p, e, 1e-3 * rng.standard_normal(T))
    nx, ny = p["nx"], p["ny"]
    w0 = 1e-3 * rng.standard_normal((ny, nx))
    wd0 = 1e-4 * rng.standard_normal((ny, nx))
    sens = np.stack([rng.integers(0, nx, ns), rng.integers(0, ny, ns)], axis=1).astype(np.int32)
    tgt = 1e-3 * rng.standard_normal((T, ns))
    return p, loaded, w0, wd0, sens, tgt
