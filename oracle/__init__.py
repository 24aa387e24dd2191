"""FP64 CPU oracle for the antiplane-shear lattice Boltzmann method with
dynamic mode III cracks (arXiv 2206.12412).

TEST INFRASTRUCTURE ONLY: the test suite, the package smoke check and the
benchmark's CPU-baseline leg are the only users.  The product path never
imports this package.  The arithmetic lives in ``lbm_oracle.c`` (plain C,
compiled here with gcc on first use); this module only marshals arguments.

A problem is described by a plain dict (see ``make_config``): lattice size,
spacing, edge kinds, material, boundary mode, crack and loads.  The same dict
is understood by the CUDA library's Python binding; nothing else is shared.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

QONE = 1 << 32  # tip fixed point: 1 dh = 2^32 units

EDGE = {"free": 0, "dirichlet": 1, "periodic": 2, "halo": 3}
EDGE_INDEX = {"left": 0, "right": 1, "bottom": 2, "top": 3}
BC = {"bounceback": 0, "macroscopic": 1}
CRACK = {"none": 0, "stationary": 1, "prescribed": 2, "kcrit": 3}
LOAD = {"zero": 0, "linear": 1, "sin2": 2, "halfsine": 3, "series": 4, "const": 5}
FLAG_CLAMPED, FLAG_UNSUPPORTED, FLAG_NONFINITE = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile lbm_oracle.c into liboracle.so next to it (gcc, -O2, with
    OpenMP where the compiler has it)."""
    with _lock:
        stale = (not os.path.exists(_LIB)) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC)
        if force or stale:
            tmp = _LIB + f".{os.getpid()}.tmp"
            cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
            # OpenMP only lets the timed CPU baseline spread the per-site loops
            # over the host's cores (orc_set_threads); without it the library
            # is the same, single-threaded
            if subprocess.call(cmd[:1] + ["-fopenmp"] + cmd[1:], stdout=subprocess.DEVNULL,
                               stderr=subprocess.DEVNULL) != 0:
                subprocess.check_call(cmd)
            os.replace(tmp, _LIB)
    return _LIB


class _Config(C.Structure):
    _fields_ = [
        ("nx", C.c_int32), ("ny", C.c_int32),
        ("dh", C.c_double), ("dt", C.c_double),
        ("edge", C.c_int32 * 4),
        ("rho", C.c_double), ("mu", C.c_double),
        ("omega", C.c_double),
        ("bc_mode", C.c_int32),
        ("crack_mode", C.c_int32),
        ("jc", C.c_int32),
        ("x_start", C.c_double), ("x_tip", C.c_double),
        ("v_rel", C.c_double), ("K_C", C.c_double), ("v_max", C.c_double),
        ("r0", C.c_double), ("r_min_fixed", C.c_double), ("fit_width", C.c_double),
        ("load_kind", C.c_int32 * 4),
        ("load_amp", C.c_double * 4), ("load_t", C.c_double * 4),
        ("load_series", C.POINTER(C.c_double) * 4),
        ("load_n", C.c_int64 * 4),
        ("hist_cap", C.c_int64),
        ("two_tips", C.c_int32), ("edge_macro", C.c_int32),
        ("q", C.c_int32), ("pad_", C.c_int32),
        ("line", C.c_int32), ("pad2_", C.c_int32),
        ("y_start", C.c_double), ("y_tip", C.c_double),
    ]


class _CrackInfo(C.Structure):
    _fields_ = [
        ("step", C.c_int64), ("tip_q", C.c_int64), ("hist_n", C.c_int64),
        ("K", C.c_double), ("v_prev", C.c_double),
        ("npairs", C.c_int32), ("flags", C.c_int32), ("n_bpoints", C.c_int32), ("pad", C.c_int32),
    ]


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        P = C.c_void_p
        d = C.POINTER(C.c_double)
        lib.orc_create.argtypes = [C.POINTER(_Config)]
        lib.orc_create.restype = P
        lib.orc_destroy.argtypes = [P]
        lib.orc_set_fields.argtypes = [P, d, d]
        lib.orc_get_fields.argtypes = [P, d, d]
        lib.orc_get_distributions.argtypes = [P, d]
        lib.orc_get_cuts.argtypes = [P, C.c_char_p, C.c_char_p]
        lib.orc_step.argtypes = [P, C.c_int64]
        lib.orc_get_crack.argtypes = [P, C.POINTER(_CrackInfo)]
        lib.orc_get_history.argtypes = [P, d, d, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                        C.POINTER(C.c_int32), C.c_int64]
        lib.orc_get_history.restype = C.c_int64
        lib.orc_get_bpoints.argtypes = [P, C.POINTER(C.c_int32), C.c_int32]
        lib.orc_get_bpoints.restype = C.c_int32
        lib.orc_get_cuts_diag.argtypes = [P, C.c_char_p, C.c_char_p]
        lib.orc_q.argtypes = [P]
        lib.orc_q.restype = C.c_int32
        lib.orc_get_edge_points.argtypes = [P, C.POINTER(C.c_int32), C.c_int32]
        lib.orc_get_edge_points.restype = C.c_int32
        lib.orc_quadratic_through.argtypes = [C.c_double] * 7
        lib.orc_quadratic_through.restype = C.c_double
        lib.orc_evaluate_K.argtypes = [P, d, C.c_int64, C.c_double, C.c_double, C.POINTER(C.c_int32)]
        lib.orc_evaluate_K.restype = C.c_double
        lib.orc_evaluate_K_left.argtypes = [P, d, C.c_int64, C.c_double, C.c_double, C.POINTER(C.c_int32)]
        lib.orc_evaluate_K_left.restype = C.c_double
        lib.orc_evaluate_K_line.argtypes = [P, d, C.c_int64, C.c_int64, C.c_double, C.c_double, C.POINTER(C.c_int32)]
        lib.orc_evaluate_K_line.restype = C.c_double
        lib.orc_tip_y.argtypes = [P]
        lib.orc_tip_y.restype = C.c_int64
        lib.orc_get_history_y.argtypes = [P, C.POINTER(C.c_int64), C.c_int64]
        lib.orc_get_history_y.restype = C.c_int64
        lib.orc_direction.argtypes = [P, d]
        lib.orc_left_tip_y.argtypes = [P]
        lib.orc_left_tip_y.restype = C.c_int64
        lib.orc_get_history_left_y.argtypes = [P, C.POINTER(C.c_int64), C.c_int64]
        lib.orc_get_history_left_y.restype = C.c_int64
        lib.orc_get_history_left.argtypes = [P, d, d, C.POINTER(C.c_int64), C.POINTER(C.c_int32),
                                             C.POINTER(C.c_int32), C.c_int64]
        lib.orc_get_history_left.restype = C.c_int64
        lib.orc_left_tip.argtypes = [P]
        lib.orc_left_tip.restype = C.c_int64
        lib.orc_equilibrium.argtypes = [C.c_double, C.c_double, C.c_double, d]
        lib.orc_macro_poly.argtypes = [C.c_double] * 5
        lib.orc_macro_poly.restype = C.c_double
        lib.orc_segments_intersect.argtypes = [C.c_int64] * 8
        lib.orc_segments_intersect.restype = C.c_int
        lib.orc_checklinks_standalone.argtypes = [
            C.c_int32, C.c_int32, C.c_char_p, C.c_char_p, C.POINTER(C.c_int32), C.c_int32,
            C.c_int64, C.c_int64, C.c_int64, C.c_int64, C.POINTER(C.c_int32), C.c_int32]
        lib.orc_checklinks_standalone.restype = C.c_int32
        lib.orc_load_value.argtypes = [P, C.c_int32, C.c_int64]
        lib.orc_load_value.restype = C.c_double
        lib.orc_collide.argtypes = [P]
        lib.orc_finish_step.argtypes = [P]
        lib.orc_fs_row.argtypes = [P, C.c_int32, d]
        lib.orc_set_halo.argtypes = [P, C.c_int32, d]
        lib.orc_halo_width.argtypes = [P]
        lib.orc_halo_width.restype = C.c_int32
        lib.orc_set_threads.argtypes = [P, C.c_int32]
        lib.orc_set_threads.restype = C.c_int32
        lib.orc_g.argtypes = [P]
        lib.orc_g.restype = C.c_double
        i32p = C.POINTER(C.c_int32)
        lib.orc_adjoint.argtypes = [C.POINTER(_Config), d, d, C.c_int64, C.c_int32, i32p, i32p, d, d, d, d, d, d]
        lib.orc_adjoint.restype = C.c_int
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_config(problem: dict):
    """Translate a problem dict into the oracle's C struct.

    Returns (struct, keepalive) -- keepalive holds the series arrays."""
    cfg = _Config()
    cfg.nx, cfg.ny = int(problem["nx"]), int(problem["ny"])
    cfg.dh, cfg.dt = float(problem.get("dh", 1.0)), float(problem.get("dt", 1.0))
    edges = problem.get("edges", ("free", "free", "dirichlet", "dirichlet"))
    for e in range(4):
        cfg.edge[e] = EDGE[edges[e]]
    cfg.rho, cfg.mu = float(problem.get("rho", 1.0)), float(problem["mu"])
    cfg.omega = float(problem.get("omega", 1.0))
    bc = problem.get("bc_mode", "bounceback")
    # "macroscopic_edges": the macroscopic rule on the crack faces and on the
    # free and Dirichlet outer edges (Sec. 3.1, Sec. 5.2)
    cfg.bc_mode = BC["macroscopic" if bc == "macroscopic_edges" else bc]
    cfg.edge_macro = 1 if bc == "macroscopic_edges" else 0
    cfg.q = {"D2Q5": 5, "D2Q9": 9}[problem.get("lattice", "D2Q5")]
    cr = problem.get("crack") or {"mode": "none"}
    cfg.crack_mode = CRACK[cr.get("mode", "none")]
    if cfg.crack_mode and "y_tip" in cr:
        # a straight crack in any direction: from (x_start, y_start) through
        # (x_tip, y_tip), growing along that direction
        cfg.line = 1
        cfg.x_start, cfg.y_start = float(cr["x_start"]), float(cr["y_start"])
        cfg.x_tip, cfg.y_tip = float(cr["x_tip"]), float(cr["y_tip"])
    elif cfg.crack_mode:
        jc = float(cr["y"]) / cfg.dh
        cfg.jc = int(round(jc))
        cfg.x_start, cfg.x_tip = float(cr.get("x_start", 0.0)), float(cr["x_tip"])
    if cfg.crack_mode:
        cfg.v_rel = float(cr.get("v_rel", 0.0))
        cfg.K_C = float(cr.get("K_C", 0.0))
        cfg.v_max = float(cr.get("v_max", 0.85))
        cfg.r0 = float(cr.get("r0", 2.0 * cfg.dh))
        cfg.r_min_fixed = float(cr.get("r_min", 0.0))
        cfg.fit_width = float(cr.get("fit_width", cfg.dh))
        cfg.two_tips = 1 if cr.get("two_tips") else 0
    keep = []
    for ld in problem.get("loads", []):
        e = EDGE_INDEX[ld["edge"]]
        cfg.load_kind[e] = LOAD[ld["kind"]]
        cfg.load_amp[e] = float(ld.get("amp", 0.0))
        cfg.load_t[e] = float(ld.get("t", 0.0))
        if ld["kind"] == "series":
            arr = np.ascontiguousarray(ld["series"], dtype=np.float64)
            keep.append(arr)
            cfg.load_series[e] = _dptr(arr)
            cfg.load_n[e] = arr.size
    cfg.hist_cap = int(problem.get("hist_cap", 1 << 16))
    return cfg, keep


class Oracle:
    """One lattice, stepped in FP64 in the paper's distribution form."""

    def __init__(self, problem: dict, threads: int = 1):
        self.lib = _load()
        self.problem = problem
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        cfg, keep = make_config(problem)
        self._cfg = cfg
        self.h = self.lib.orc_create(C.byref(cfg))
        if not self.h:
            raise ValueError("oracle rejected the configuration")
        del keep  # the library copies series at create
        # threads of the per-site loops (results do not depend on it)
        self.threads = int(self.lib.orc_set_threads(self.h, int(threads)))

    def close(self):
        if getattr(self, "h", None):
            self.lib.orc_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()

    def set_fields(self, w: np.ndarray, wdot: np.ndarray):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.ny, self.nx)
        wd = np.ascontiguousarray(wdot, dtype=np.float64).reshape(self.ny, self.nx)
        self.lib.orc_set_fields(self.h, _dptr(w), _dptr(wd))

    def fields(self):
        w = np.empty((self.ny, self.nx))
        wd = np.empty((self.ny, self.nx))
        self.lib.orc_get_fields(self.h, _dptr(w), _dptr(wd))
        return w, wd

    def distributions(self):
        f = np.empty((self.lib.orc_q(self.h), self.ny, self.nx))
        self.lib.orc_get_distributions(self.h, _dptr(f))
        return f

    def step(self, n: int = 1):
        self.lib.orc_step(self.h, int(n))

    # row slabs (bottom / top edges of kind "halo"): a step is collide(),
    # then the exchange of the post-collision rows that cross the slab's
    # boundaries (fs_row -> the neighbour's set_halo), then finish_step()
    def collide(self):
        self.lib.orc_collide(self.h)

    def fs_row(self, side: int) -> np.ndarray:
        """Post-collision values leaving across the bottom (side 0) or top (1)
        edge: halo_width() rows of nx (D2Q5: the y direction; D2Q9: it and
        the two diagonals)."""
        out = np.empty(self.nx * self.lib.orc_halo_width(self.h))
        self.lib.orc_fs_row(self.h, int(side), _dptr(out))
        return out

    def set_halo(self, side: int, row):
        """The neighbour's values arriving across the bottom (side 0) or top (1) edge."""
        r = np.ascontiguousarray(row, dtype=np.float64)
        assert r.size == self.nx * self.lib.orc_halo_width(self.h)
        self.lib.orc_set_halo(self.h, int(side), _dptr(r))

    def finish_step(self):
        self.lib.orc_finish_step(self.h)

    def cuts(self):
        """(cut_h, cut_v) as (ny, nx) uint8: link (i,j)-(i+1,j) / (i,j)-(i,j+1) severed."""
        ch = np.zeros((self.ny, self.nx), np.uint8)
        cv = np.zeros((self.ny, self.nx), np.uint8)
        self.lib.orc_get_cuts(self.h, ch.ctypes.data_as(C.c_char_p), cv.ctypes.data_as(C.c_char_p))
        return ch, cv

    def cuts_diag(self):
        """D2Q9: (cut_d1, cut_d2) as (ny, nx) uint8: links (i,j)-(i+1,j+1) and
        (i+1,j)-(i,j+1) severed (flags at (i,j))."""
        d1 = np.zeros((self.ny, self.nx), np.uint8)
        d2 = np.zeros((self.ny, self.nx), np.uint8)
        self.lib.orc_get_cuts_diag(self.h, d1.ctypes.data_as(C.c_char_p), d2.ctypes.data_as(C.c_char_p))
        return d1, d2

    def crack(self) -> dict:
        info = _CrackInfo()
        self.lib.orc_get_crack(self.h, C.byref(info))
        return {k: getattr(info, k) for k, _ in _CrackInfo._fields_ if k != "pad"}

    def history(self) -> dict:
        cap = int(self.problem.get("hist_cap", 1 << 16))
        K = np.zeros(cap); v = np.zeros(cap)
        tip = np.zeros(cap, np.int64); npairs = np.zeros(cap, np.int32); grew = np.zeros(cap, np.int32)
        n = self.lib.orc_get_history(self.h, _dptr(K), _dptr(v), tip.ctypes.data_as(C.POINTER(C.c_int64)),
                                     npairs.ctypes.data_as(C.POINTER(C.c_int32)),
                                     grew.ctypes.data_as(C.POINTER(C.c_int32)), cap)
        out = {"K": K[:n], "v": v[:n], "tip_q": tip[:n], "npairs": npairs[:n], "grew": grew[:n]}
        if self._cfg.line:
            ty = np.zeros(cap, np.int64)
            self.lib.orc_get_history_y(self.h, ty.ctypes.data_as(C.POINTER(C.c_int64)), cap)
            out["tip_yq"] = ty[:n]
        return out

    def tip_y_q(self) -> int:
        """y of the tip (units of 2^-32 dh); the crack along +x keeps y = jc dh."""
        return int(self.lib.orc_tip_y(self.h))

    def direction(self):
        """Unit direction of growth (c_x, c_y)."""
        out = np.zeros(2)
        self.lib.orc_direction(self.h, _dptr(out))
        return float(out[0]), float(out[1])

    def evaluate_K_line(self, w: np.ndarray, tip_xq: int, tip_yq: int, r_min: float, fit_width: float):
        """K of a crack in any direction at the tip (tip_xq, tip_yq), from the
        fields w and the oracle's current cut mask."""
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.ny, self.nx)
        npairs = C.c_int32(0)
        K = self.lib.orc_evaluate_K_line(self.h, _dptr(w), int(tip_xq), int(tip_yq), float(r_min), float(fit_width),
                                         C.byref(npairs))
        return K, npairs.value

    def history_left(self) -> dict:
        """Per-step record of the left end of a two-tip crack."""
        cap = int(self.problem.get("hist_cap", 1 << 16))
        K = np.zeros(cap); v = np.zeros(cap)
        tip = np.zeros(cap, np.int64); npairs = np.zeros(cap, np.int32); grew = np.zeros(cap, np.int32)
        n = self.lib.orc_get_history_left(self.h, _dptr(K), _dptr(v), tip.ctypes.data_as(C.POINTER(C.c_int64)),
                                          npairs.ctypes.data_as(C.POINTER(C.c_int32)),
                                          grew.ctypes.data_as(C.POINTER(C.c_int32)), cap)
        out = {"K": K[:n], "v": v[:n], "tip_q": tip[:n], "npairs": npairs[:n], "grew": grew[:n]}
        if self._cfg.line:
            ty = np.zeros(cap, np.int64)
            self.lib.orc_get_history_left_y(self.h, ty.ctypes.data_as(C.POINTER(C.c_int64)), cap)
            out["tip_yq"] = ty[:n]
        return out

    def left_tip_y_q(self) -> int:
        return int(self.lib.orc_left_tip_y(self.h))

    def left_tip_q(self) -> int:
        return int(self.lib.orc_left_tip(self.h))

    def evaluate_K_left(self, w: np.ndarray, tip_q: int, r_min: float, fit_width: float):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.ny, self.nx)
        npairs = C.c_int32(0)
        K = self.lib.orc_evaluate_K_left(self.h, _dptr(w), int(tip_q), float(r_min), float(fit_width), C.byref(npairs))
        return K, npairs.value

    def bpoints(self) -> np.ndarray:
        cap = 4 * (self.nx + self.ny) + 64
        out = np.zeros(cap, np.int32)
        n = self.lib.orc_get_bpoints(self.h, out.ctypes.data_as(C.POINTER(C.c_int32)), cap)
        return out[:n]

    def edge_points(self) -> np.ndarray:
        """Outer-edge boundary points of the macroscopic rule: rows (site,
        x_I site, x_II site, rule (0 free, 1 Dirichlet), edge index)."""
        cap = 2 * (self.nx + self.ny)
        out = np.zeros((cap, 5), np.int32)
        n = self.lib.orc_get_edge_points(self.h, out.ctypes.data_as(C.POINTER(C.c_int32)), cap)
        return out[:n]

    def flags(self) -> int:
        return int(self.crack()["flags"])

    def evaluate_K(self, w: np.ndarray, tip_q: int, r_min: float, fit_width: float):
        w = np.ascontiguousarray(w, dtype=np.float64).reshape(self.ny, self.nx)
        npairs = C.c_int32(0)
        K = self.lib.orc_evaluate_K(self.h, _dptr(w), int(tip_q), float(r_min), float(fit_width), C.byref(npairs))
        return K, npairs.value

    def load_value(self, edge: str, n: int) -> float:
        return self.lib.orc_load_value(self.h, EDGE_INDEX[edge], int(n))

    @property
    def g(self) -> float:
        return self.lib.orc_g(self.h)


def equilibrium(w: float, wdot: float, g: float) -> np.ndarray:
    out = np.zeros(5)
    _load().orc_equilibrium(w, wdot, g, _dptr(out))
    return out


def macro_poly(sB, sI, sII, wI, wII) -> float:
    return _load().orc_macro_poly(sB, sI, sII, wI, wII)


def quadratic_through(s0, v0, s1, v1, s2, v2, x) -> float:
    """The quadratic polynomial through three points, evaluated at x."""
    return _load().orc_quadratic_through(s0, v0, s1, v1, s2, v2, x)


def segments_intersect(p1, p2, q1, q2) -> bool:
    return bool(_load().orc_segments_intersect(*p1, *p2, *q1, *q2))


def checklinks(nx, ny, cut_h, cut_v, bprev, seg_a, seg_b, nmax=256):
    """Alg. 1 CheckLinks on a bare lattice.  cut_h / cut_v are (ny, nx) uint8
    arrays updated in place; returns the sorted new boundary points."""
    assert cut_h.dtype == np.uint8 and cut_h.flags.c_contiguous
    assert cut_v.dtype == np.uint8 and cut_v.flags.c_contiguous
    bp = np.ascontiguousarray(bprev, dtype=np.int32)
    out = np.zeros(nmax, np.int32)
    n = _load().orc_checklinks_standalone(
        nx, ny, cut_h.ctypes.data_as(C.c_char_p), cut_v.ctypes.data_as(C.c_char_p),
        bp.ctypes.data_as(C.POINTER(C.c_int32)), bp.size,
        int(seg_a[0]), int(seg_a[1]), int(seg_b[0]), int(seg_b[1]),
        out.ctypes.data_as(C.POINTER(C.c_int32)), nmax)
    return np.sort(out[:n])


def adjoint(problem: dict, n_steps: int, sensors, targets, w0=None, wd0=None, grad: bool = True) -> dict:
    """Sensor misfit L = sum_{n=1..T} sum_s (w^n_s - target[n-1, s])^2 of a
    T-step oracle run from (w0, wd0), and (if grad) its gradient by the
    transposed steps under the run's own cut schedule.

    sensors: (ns, 2) integer (i, j) sites; targets: (T, ns).  Returns a dict
    with loss, trace (T, ns) of w at the sensors, and if grad: dload (4, T)
    (dL/dw*_e(t_n), edges left/right/bottom/top), dw0 and dwd0 (ny, nx)."""
    lib = _load()
    cfg, keep = make_config(problem)
    nx, ny = int(problem["nx"]), int(problem["ny"])
    T = int(n_steps)
    sens = np.ascontiguousarray(np.asarray(sensors, dtype=np.int32).reshape(-1, 2))
    si = np.ascontiguousarray(sens[:, 0])
    sj = np.ascontiguousarray(sens[:, 1])
    ns = sens.shape[0]
    tgt = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(T, ns))
    zero = np.zeros((ny, nx))
    w0a = np.ascontiguousarray(zero if w0 is None else np.asarray(w0, np.float64).reshape(ny, nx))
    wd0a = np.ascontiguousarray(zero if wd0 is None else np.asarray(wd0, np.float64).reshape(ny, nx))
    loss = C.c_double(0.0)
    trace = np.zeros((T, ns))
    out = {}
    null = C.POINTER(C.c_double)()
    if grad:
        dload = np.zeros((4, T))
        dw0 = np.zeros((ny, nx))
        dwd0 = np.zeros((ny, nx))
        args = (_dptr(dload), _dptr(dw0), _dptr(dwd0))
    else:
        args = (null, null, null)
    i32 = C.POINTER(C.c_int32)
    rc = lib.orc_adjoint(C.byref(cfg), _dptr(w0a), _dptr(wd0a), T, ns, si.ctypes.data_as(i32),
                         sj.ctypes.data_as(i32), _dptr(tgt), C.byref(loss), _dptr(trace), *args)
    del keep
    if rc != 0:
        raise ValueError("oracle rejected the adjoint problem")
    out["loss"] = loss.value
    out["trace"] = trace
    if grad:
        out["dload"], out["dw0"], out["dwd0"] = dload, dw0, dwd0
    return out
