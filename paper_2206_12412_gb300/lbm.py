"""Python binding of liblbm.so: the C-ABI calls under their own names, plus a
small ``Lattice`` convenience class driven by a problem dict.

Argument marshalling only -- every step of the method runs in the library's
CUDA kernels.  There is no CPU path: if the library cannot be loaded, every
call raises.  Device memory comes from PyTorch's caching allocator (passed to
``lbm_create`` as the allocator callbacks) and work is enqueued on the current
PyTorch CUDA stream unless another stream is given.
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import _abi as A

_lib = None
_lib_lock = threading.Lock()


class LbmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{A.STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


def library_path() -> str:
    from .build import LIB_PATH
    return LIB_PATH


def load_library():
    """Load liblbm.so (building it in-tree first if it is missing or stale)."""
    global _lib
    with _lib_lock:
        if _lib is None:
            from . import build as _build
            if _build.is_stale():
                _build.build()
            lib = C.CDLL(_build.LIB_PATH)
            for name, (res, args) in A.PROTOTYPES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != A.LBM_OK:
        msg = load_library().lbm_last_error()
        raise LbmError(status, msg.decode() if msg else "")


# ----------------------------------------------------------- C-ABI calls

def lbm_create(grid: A.Grid, lattice: A.Lattice_, material: A.Material, crack: A.Crack | None,
               loads, stream: int = 0, allocator: A.Allocator | None = None) -> int:
    lib = load_library()
    n = len(loads)
    arr = (A.Loading * max(n, 1))(*loads) if n else None
    out = C.c_void_p()
    _check(lib.lbm_create(C.byref(grid), C.byref(lattice), C.byref(material),
                          C.byref(crack) if crack is not None else None,
                          arr, n, C.c_void_p(stream), C.byref(allocator) if allocator is not None else None,
                          C.byref(out)))
    return out.value


def lbm_create_line(grid: A.Grid, lattice: A.Lattice_, material: A.Material, crack: A.CrackLine,
                    loads, stream: int = 0, allocator: A.Allocator | None = None) -> int:
    lib = load_library()
    n = len(loads)
    arr = (A.Loading * max(n, 1))(*loads) if n else None
    out = C.c_void_p()
    _check(lib.lbm_create_line(C.byref(grid), C.byref(lattice), C.byref(material), C.byref(crack),
                               arr, n, C.c_void_p(stream), C.byref(allocator) if allocator is not None else None,
                               C.byref(out)))
    return out.value


def lbm_line_tip(h: int, cap: int = 0, left: bool = False):
    """(x_q, y_q) of the tip (left: the growing start of a two-tip crack) of a
    crack in any direction and the y of its last `cap` records."""
    x, y, nw = C.c_int64(0), C.c_int64(0), C.c_int64(0)
    ys = np.zeros(max(cap, 1), np.int64)
    fn = load_library().lbm_line_tip_left if left else load_library().lbm_line_tip
    _check(fn(C.c_void_p(h), C.byref(x), C.byref(y), ys.ctypes.data_as(C.POINTER(C.c_int64)), cap, C.byref(nw)))
    return x.value, y.value, ys[:nw.value]


def lbm_step(h: int, n: int):
    _check(load_library().lbm_step(C.c_void_p(h), int(n)))


def lbm_fields(h: int, which: int, dst_ptr: int, on_device: bool, dtype: int):
    _check(load_library().lbm_fields(C.c_void_p(h), which, C.c_void_p(dst_ptr), int(bool(on_device)), dtype))


def lbm_set_fields(h: int, which: int, src_ptr: int, on_device: bool, dtype: int):
    _check(load_library().lbm_set_fields(C.c_void_p(h), which, C.c_void_p(src_ptr), int(bool(on_device)), dtype))


def lbm_fields_strided(h: int, which: int, dst_ptr: int, on_device: bool, dtype: int, row_stride: int):
    _check(load_library().lbm_fields_strided(C.c_void_p(h), which, C.c_void_p(dst_ptr), int(bool(on_device)), dtype,
                                             int(row_stride)))


def lbm_set_fields_strided(h: int, which: int, src_ptr: int, on_device: bool, dtype: int, row_stride: int):
    _check(load_library().lbm_set_fields_strided(C.c_void_p(h), which, C.c_void_p(src_ptr), int(bool(on_device)),
                                                 dtype, int(row_stride)))


def lbm_cut_mask(h: int, which: int, dst: np.ndarray):
    assert dst.dtype == np.uint32 and dst.flags.c_contiguous
    _check(load_library().lbm_cut_mask(C.c_void_p(h), which, dst.ctypes.data_as(C.POINTER(C.c_uint32)), dst.size))


def lbm_crack_state(h: int, cap: int = 0, left: bool = False):
    """Crack state and last `cap` records of the right end (left: the left
    end of a two-tip crack)."""
    st = A.CrackStateT()
    K = np.zeros(max(cap, 1)); v = np.zeros(max(cap, 1))
    tip = np.zeros(max(cap, 1), np.int64); np_ = np.zeros(max(cap, 1), np.int32)
    nw = C.c_int64(0)
    d = C.POINTER(C.c_double)
    fn = load_library().lbm_crack_state_left if left else load_library().lbm_crack_state
    _check(fn(
        C.c_void_p(h), C.byref(st), K.ctypes.data_as(d), v.ctypes.data_as(d),
        tip.ctypes.data_as(C.POINTER(C.c_int64)), np_.ctypes.data_as(C.POINTER(C.c_int32)), cap, C.byref(nw)))
    n = nw.value
    return st, {"K": K[:n], "v": v[:n], "tip_q": tip[:n], "npairs": np_[:n]}


def lbm_sync(h: int):
    _check(load_library().lbm_sync(C.c_void_p(h)))


def lbm_set_stream(h: int, stream: int):
    _check(load_library().lbm_set_stream(C.c_void_p(h), C.c_void_p(stream)))


def lbm_set_launch(h: int, band_rows: int):
    _check(load_library().lbm_set_launch(C.c_void_p(h), int(band_rows)))


def lbm_set_face_solve(h: int, mode: int) -> bool:
    ch = C.c_int32()
    _check(load_library().lbm_set_face_solve(C.c_void_p(h), int(mode), C.byref(ch)))
    return bool(ch.value)


def lbm_get_launch(h: int) -> dict:
    r, c, t, s = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
    _check(load_library().lbm_get_launch(C.c_void_p(h), C.byref(r), C.byref(c), C.byref(t), C.byref(s)))
    return {"band_rows": r.value, "ctas": c.value, "threads": t.value, "ctas_per_sm": s.value}


def lbm_set_profiling(h: int, enable: bool):
    _check(load_library().lbm_set_profiling(C.c_void_p(h), int(bool(enable))))


def lbm_profile_read(h: int, reset: bool = False):
    bm, cm = C.c_double(), C.c_double()
    nb, nc = C.c_int64(), C.c_int64()
    _check(load_library().lbm_profile_read(C.c_void_p(h), C.byref(bm), C.byref(nb), C.byref(cm), C.byref(nc),
                                           int(bool(reset))))
    return {"step_ms": bm.value, "n_step": nb.value, "finalize_ms": cm.value, "n_finalize": nc.value}


def lbm_set_wd_scale(h: int, scale: float):
    _check(load_library().lbm_set_wd_scale(C.c_void_p(h), float(scale)))


def lbm_get_wd_scale(h: int) -> float:
    v = C.c_double()
    _check(load_library().lbm_get_wd_scale(C.c_void_p(h), C.byref(v)))
    return v.value


def lbm_device_bytes(h: int) -> int:
    b = C.c_int64()
    _check(load_library().lbm_device_bytes(C.c_void_p(h), C.byref(b)))
    return b.value


def lbm_save(h: int, path: str):
    _check(load_library().lbm_save(C.c_void_p(h), os.fsencode(path)))


def lbm_load(h: int, path: str):
    _check(load_library().lbm_load(C.c_void_p(h), os.fsencode(path)))


def lbm_destroy(h: int):
    if h:
        load_library().lbm_destroy(C.c_void_p(h))


def lbm_reset(h: int):
    _check(load_library().lbm_reset(C.c_void_p(h)))


def make_loading(edge: str, kind: str, series=None, amp: float = 0.0, t_ramp: float = 0.0):
    """(lbm_loading struct, keepalive) for one edge."""
    L = A.Loading()
    L.edge = A.EDGE_INDEX[edge]
    L.kind = A.LOAD[kind]
    L.amp = float(amp)
    L.t_ramp = float(t_ramp)
    arr = None
    if kind == "series":
        arr = np.ascontiguousarray(series, dtype=np.float64)
        L.series = arr.ctypes.data_as(C.POINTER(C.c_double))
        L.n_series = arr.size
    return L, arr


def lbm_set_loading(h: int, edge: str, kind: str, series=None, amp: float = 0.0, t_ramp: float = 0.0):
    L, keep = make_loading(edge, kind, series, amp, t_ramp)
    _check(load_library().lbm_set_loading(C.c_void_p(h), C.byref(L)))
    del keep


def lbm_wdot_to_host_noalloc(h: int, dst: np.ndarray):
    """16-bit wdot plane -> dst (float32, nx * ny), through the library's fixed
    conversion array (no allocation)."""
    assert dst.dtype == np.float32 and dst.flags.c_contiguous
    _check(load_library().lbm_wdot_to_host_noalloc(C.c_void_p(h), dst.ctypes.data_as(C.POINTER(C.c_float)),
                                                   dst.size))


def lbm_last_error() -> str:
    return load_library().lbm_last_error().decode()


# ------------------------------------------------- problem dict -> structs

def make_structs(problem: dict, storage: str = "f32"):
    """C structs for a problem dict (the same dict the oracle reads)."""
    g = A.Grid()
    g.nx, g.ny = int(problem["nx"]), int(problem["ny"])
    g.dh, g.dt = float(problem.get("dh", 1.0)), float(problem.get("dt", 1.0))
    edges = problem.get("edges", ("free", "free", "dirichlet", "dirichlet"))
    for e in range(4):
        g.edge[e] = A.EDGE[edges[e]]
    lat = A.Lattice_()
    lat.velocity_set, lat.form = A.VELOCITY_SET[problem.get("lattice", "D2Q5")], 0
    lat.omega = float(problem.get("omega", 1.0))
    lat.storage = A.STORAGE[storage]
    lat.bc_mode = A.BC[problem.get("bc_mode", "bounceback")]
    mat = A.Material()
    mat.rho, mat.mu = float(problem.get("rho", 1.0)), float(problem["mu"])
    c = problem.get("crack") or {"mode": "none"}
    line = "y_tip" in c                       # a straight crack in any direction (lbm_create_line)
    cr = A.CrackLine() if line else A.Crack()
    cr.mode = A.CRACK[c.get("mode", "none")]
    if cr.mode:
        if line:
            cr.x_start, cr.y_start = float(c["x_start"]), float(c["y_start"])
            cr.x_tip, cr.y_tip = float(c["x_tip"]), float(c["y_tip"])
        else:
            cr.y = float(c["y"])
            cr.x_start, cr.x_tip = float(c.get("x_start", 0.0)), float(c["x_tip"])
        cr.two_tips = 1 if c.get("two_tips") else 0
        cr.v_rel = float(c.get("v_rel", 0.0))
        cr.K_C = float(c.get("K_C", 0.0))
        cr.v_max = float(c.get("v_max", 0.85))
        cr.r0 = float(c.get("r0", 2.0 * g.dh))
        cr.r_min = float(c.get("r_min", 0.0))
        cr.fit_width = float(c.get("fit_width", g.dh))
        cr.hist_cap = int(problem.get("hist_cap", 1 << 16))
    loads = []
    keep = []
    for ld in problem.get("loads", []):
        L = A.Loading()
        L.edge = A.EDGE_INDEX[ld["edge"]]
        L.kind = A.LOAD[ld["kind"]]
        L.amp = float(ld.get("amp", 0.0))
        L.t_ramp = float(ld.get("t", 0.0))
        if ld["kind"] == "series":
            arr = np.ascontiguousarray(ld["series"], dtype=np.float64)
            keep.append(arr)
            L.series = arr.ctypes.data_as(C.POINTER(C.c_double))
            L.n_series = arr.size
        loads.append(L)
    return g, lat, mat, cr, loads, keep


class TorchAllocator:
    """lbm_allocator callbacks backed by torch's CUDA caching allocator."""

    def __init__(self, stream: int):
        import torch
        self._torch = torch
        self._stream = stream

        def _alloc(nbytes, ctx):
            try:
                return self._torch.cuda.caching_allocator_alloc(int(nbytes), stream=self._stream or None)
            except Exception:
                return None

        def _release(ptr, ctx):
            if ptr:
                self._torch.cuda.caching_allocator_delete(ptr)

        self._fa = A.ALLOC_FN(_alloc)
        self._fr = A.RELEASE_FN(_release)
        self.struct = A.Allocator(self._fa, self._fr, None)


class Lattice:
    """One lattice handle on the current CUDA device.

    problem: dict with nx, ny, dh, dt, edges, rho, mu, omega, bc_mode, crack,
    loads, hist_cap (see ``workloads``).  storage: "f32" or "f64"."""

    def __init__(self, problem: dict, storage: str = "f32", stream=None, torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.problem = problem
        self.storage = storage
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        self.np_dtype = np.float64 if storage == "f64" else np.float32
        self.torch_dtype = torch.float64 if storage == "f64" else torch.float32
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream_obj = stream
        self.stream = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
        g, lat, mat, cr, loads, keep = make_structs(problem, storage)
        self._alloc = TorchAllocator(self.stream) if torch_allocator else None
        self.line = isinstance(cr, A.CrackLine)
        if self.line:
            self.h = lbm_create_line(g, lat, mat, cr, loads, self.stream, self._alloc.struct if self._alloc else None)
        else:
            self.h = lbm_create(g, lat, mat, cr if cr.mode else None, loads, self.stream,
                                self._alloc.struct if self._alloc else None)
        del keep

    @property
    def dtype_code(self) -> int:
        """Exchange dtype of the fields: LBM_F64 for f64 storage, LBM_F32 otherwise."""
        return A.STORAGE["f64"] if self.storage == "f64" else A.STORAGE["f32"]

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def step(self, n: int = 1):
        lbm_step(self.h, n)

    def set_launch(self, band_rows: int):
        lbm_set_launch(self.h, band_rows)

    def set_bulk(self, enable: bool = True):
        """Stage the interior CTAs' rows by bulk asynchronous copies
        (lbm_set_bulk); same results."""
        _check(load_library().lbm_set_bulk(C.c_void_p(self.h), 1 if enable else 0))

    def set_chained(self, enable: bool = True):
        """Launch the kernels of consecutive steps chained by programmatic
        dependent launch (lbm_set_chained; the default) or plainly; same
        results."""
        _check(load_library().lbm_set_chained(C.c_void_p(self.h), 1 if enable else 0))

    def set_face_solve(self, mode: int) -> bool:
        """0: the chunked solve of the line crack's macroscopic faces where
        the coupling allows it, 1: the one-CTA solve; returns whether the
        chunked one runs."""
        return lbm_set_face_solve(self.h, mode)

    def launch(self):
        return lbm_get_launch(self.h)

    def set_fields(self, w=None, wdot=None):
        for which, arr in (("w", w), ("wdot", wdot)):
            if arr is None:
                continue
            if isinstance(arr, self.torch.Tensor) and arr.is_cuda:
                t = arr.to(self.torch_dtype).contiguous()
                assert t.numel() == self.nx * self.ny
                lbm_set_fields(self.h, A.FIELD[which], t.data_ptr(), True, self.dtype_code)
                self.torch.cuda.current_stream().synchronize()
            else:
                a = np.ascontiguousarray(np.asarray(arr, dtype=self.np_dtype).reshape(self.ny, self.nx))
                lbm_set_fields(self.h, A.FIELD[which], a.ctypes.data, False, self.dtype_code)

    def fields(self):
        """(w, wdot) as host numpy arrays of shape (ny, nx)."""
        out = []
        for which in ("w", "wdot"):
            a = np.empty((self.ny, self.nx), self.np_dtype)
            lbm_fields(self.h, A.FIELD[which], a.ctypes.data, False, self.dtype_code)
            out.append(a)
        return tuple(out)

    def fields_device(self):
        """(w, wdot) as CUDA tensors (copies, enqueued on the handle's stream)."""
        out = []
        for which in ("w", "wdot"):
            t = self.torch.empty((self.ny, self.nx), dtype=self.torch_dtype, device="cuda")
            lbm_fields(self.h, A.FIELD[which], t.data_ptr(), True, self.dtype_code)
            out.append(t)
        return tuple(out)

    def cut_mask(self, which: str = "v") -> np.ndarray:
        """Severed links as a (ny, nx) bool array (H: link to i+1, V: link to j+1)."""
        words = (self.nx + 31) // 32
        raw = np.zeros(self.ny * words, np.uint32)
        lbm_cut_mask(self.h, A.MASK[which], raw)
        bits = np.unpackbits(raw.view(np.uint8).reshape(self.ny, words * 4), axis=1, bitorder="little")
        return bits[:, : self.nx].astype(bool)

    def crack_state(self, cap: int = 0):
        st, hist = lbm_crack_state(self.h, cap)
        d = {k: getattr(st, k) for k, _ in A.CrackStateT._fields_}
        return (d, hist) if cap else d

    def history(self, cap: int | None = None) -> dict:
        """Per-step K, v, tip (x; with "tip_yq" the y of a crack in any
        direction) and pairs, oldest first."""
        if cap is None:
            cap = int(self.problem.get("hist_cap", 1 << 16))
        h = lbm_crack_state(self.h, cap)[1]
        if getattr(self, "line", False):
            h["tip_yq"] = lbm_line_tip(self.h, cap)[2]
        return h

    def tip_q(self):
        """(x, y) of the tip of a crack in any direction, units of 2^-32 dh."""
        x, y, _ = lbm_line_tip(self.h)
        return x, y

    def crack_state_left(self):
        """State of the left end of a two-tip crack."""
        st, _ = lbm_crack_state(self.h, 0, left=True)
        return {k: getattr(st, k) for k, _ in A.CrackStateT._fields_}

    def history_left(self, cap: int | None = None) -> dict:
        if cap is None:
            cap = int(self.problem.get("hist_cap", 1 << 16))
        h = lbm_crack_state(self.h, cap, left=True)[1]
        if getattr(self, "line", False):
            h["tip_yq"] = lbm_line_tip(self.h, cap, left=True)[2]
        return h

    def tip_q_left(self):
        """(x, y) of the growing start of a two-tip crack in any direction."""
        x, y, _ = lbm_line_tip(self.h, left=True)
        return x, y

    def sync(self):
        lbm_sync(self.h)

    def set_profiling(self, enable: bool = True):
        lbm_set_profiling(self.h, enable)

    def profile(self, reset: bool = False) -> dict:
        return lbm_profile_read(self.h, reset)

    def set_wd_scale(self, scale: float):
        lbm_set_wd_scale(self.h, scale)

    def wd_scale(self) -> float:
        return lbm_get_wd_scale(self.h)

    def device_bytes(self) -> int:
        return lbm_device_bytes(self.h)

    def save(self, path: str):
        """Write the lattice's whole state to a checkpoint file."""
        lbm_save(self.h, path)

    def load(self, path: str):
        """Read a checkpoint written by a lattice of the same problem."""
        lbm_load(self.h, path)

    def reset(self):
        """Back to step 0: zero fields, the initial crack, empty history."""
        lbm_reset(self.h)

    def set_loading(self, edge: str, kind: str, series=None, amp: float = 0.0, t_ramp: float = 0.0):
        """Replace one edge's loading (a series no longer than at creation)."""
        if series is not None and isinstance(series, self.torch.Tensor):
            series = series.detach().to("cpu", self.torch.float64).numpy()
        lbm_set_loading(self.h, edge, kind, series, amp, t_ramp)


# ----------------------------------------------------------------- batches

def lbm_batch_create(handles, band_rows: int = 0, allocator: A.Allocator | None = None) -> int:
    arr = (C.c_void_p * len(handles))(*handles)
    out = C.c_void_p()
    _check(load_library().lbm_batch_create(arr, len(handles), int(band_rows),
                                           C.byref(allocator) if allocator is not None else None, C.byref(out)))
    return out.value


def lbm_batch_step(b: int, n: int):
    _check(load_library().lbm_batch_step(C.c_void_p(b), int(n)))


def lbm_batch_info(b: int):
    nl, ct = C.c_int32(), C.c_int32()
    _check(load_library().lbm_batch_info(C.c_void_p(b), C.byref(nl), C.byref(ct)))
    return {"lattices": nl.value, "ctas": ct.value}


def lbm_batch_set_shape(b: int, threads: int, band_rows: int):
    _check(load_library().lbm_batch_set_shape(C.c_void_p(b), int(threads), int(band_rows)))


def lbm_batch_get_shape(b: int):
    t, r = C.c_int32(), C.c_int32()
    _check(load_library().lbm_batch_get_shape(C.c_void_p(b), C.byref(t), C.byref(r)))
    return {"threads": t.value, "band_rows": r.value}


def lbm_batch_set_lookahead(b: int, rows: int):
    _check(load_library().lbm_batch_set_lookahead(C.c_void_p(b), int(rows)))


def lbm_batch_get_lookahead(b: int) -> int:
    r = C.c_int32()
    _check(load_library().lbm_batch_get_lookahead(C.c_void_p(b), C.byref(r)))
    return r.value


def lbm_batch_tune(b: int, trial_steps: int = 8):
    t, r, us, fc = C.c_int32(), C.c_int32(), C.c_double(), C.c_int32()
    _check(load_library().lbm_batch_tune(C.c_void_p(b), int(trial_steps), C.byref(t), C.byref(r), C.byref(us),
                                         C.byref(fc)))
    return {"threads": t.value, "band_rows": r.value, "lookahead": lbm_batch_get_lookahead(b),
            "us_per_step": us.value, "from_cache": bool(fc.value)}


def lbm_batch_set_persistent(b: int, enable: bool, budget_cycles: int = 0):
    _check(load_library().lbm_batch_set_persistent(C.c_void_p(b), 1 if enable else 0, int(budget_cycles)))


def lbm_barrier_probe(ctas: int, expected: int, budget_cycles: int, stream: int = 0):
    _check(load_library().lbm_barrier_probe(int(ctas), int(expected), int(budget_cycles), C.c_void_p(stream)))


def lbm_batch_destroy(b: int):
    if b:
        load_library().lbm_batch_destroy(C.c_void_p(b))


def lbm_create_batch(problems, storage: str = "f32", stream: int = 0, allocator: A.Allocator | None = None,
                     band_rows: int = 0) -> int:
    """lbm_create_batch over problem dicts (one storage for all): the batch
    owns its lattices."""
    n = len(problems)
    grids, lats, mats, cracks = (A.Grid * n)(), (A.Lattice_ * n)(), (A.Material * n)(), (A.Crack * n)()
    load_arrs, nloads, keep = [], (C.c_int32 * n)(), []
    for i, p in enumerate(problems):
        g, lat, mat, cr, loads, k = make_structs(p, storage)
        if isinstance(cr, A.CrackLine):
            raise ValueError("lbm_create_batch takes cracks along +x (lbm_crack)")
        grids[i], lats[i], mats[i], cracks[i] = g, lat, mat, cr
        arr = (A.Loading * max(len(loads), 1))(*loads)
        load_arrs.append(C.cast(arr, C.POINTER(A.Loading)))
        nloads[i] = len(loads)
        keep += [arr, k]
    lptrs = (C.POINTER(A.Loading) * n)(*load_arrs)
    out = C.c_void_p()
    _check(load_library().lbm_create_batch(n, grids, lats, mats, cracks, lptrs, nloads, C.c_void_p(stream),
                                           C.byref(allocator) if allocator is not None else None, int(band_rows),
                                           C.byref(out)))
    del keep
    return out.value


def lbm_batch_member(b: int, i: int) -> int:
    out = C.c_void_p()
    _check(load_library().lbm_batch_member(C.c_void_p(b), int(i), C.byref(out)))
    return out.value


class Batch:
    """Several Lattice objects advanced together, one kernel launch per step."""

    def __init__(self, lattices, band_rows: int = 0, torch_allocator: bool = True):
        self.lattices = list(lattices)
        self._alloc = TorchAllocator(self.lattices[0].stream) if torch_allocator else None
        self.b = lbm_batch_create([l.h for l in self.lattices], band_rows,
                                  self._alloc.struct if self._alloc else None)

    def step(self, n: int = 1):
        lbm_batch_step(self.b, n)

    def info(self) -> dict:
        return dict(lbm_batch_info(self.b), **lbm_batch_get_shape(self.b), lookahead=lbm_batch_get_lookahead(self.b))

    def set_shape(self, threads: int, band_rows: int):
        lbm_batch_set_shape(self.b, threads, band_rows)

    def set_lookahead(self, rows: int):
        """Rows of loads the march keeps in flight ahead (1 or 2)."""
        lbm_batch_set_lookahead(self.b, rows)

    def set_chained(self, enable: bool = True):
        """Chained launches of the batched step (lbm_batch_set_chained)."""
        _check(load_library().lbm_batch_set_chained(C.c_void_p(self.b), 1 if enable else 0))

    def set_persistent(self, enable: bool = True, budget_cycles: int = 0):
        """One cooperative launch per lbm_batch_step call (grid barrier
        between steps, each wait bounded by budget_cycles)."""
        lbm_batch_set_persistent(self.b, enable, budget_cycles)

    def tune(self, trial_steps: int = 8) -> dict:
        """Pick the fastest launch shape (lbm_batch_tune); the lattices'
        state is left as it was."""
        return lbm_batch_tune(self.b, trial_steps)

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- adjoint

def lbm_tape_create(h: int, sensors, n_steps: int, checkpoint_every: int = 0,
                    allocator: A.Allocator | None = None) -> int:
    sens = np.ascontiguousarray(np.asarray(sensors, dtype=np.int32).reshape(-1, 2))
    out = C.c_void_p()
    _check(load_library().lbm_tape_create(C.c_void_p(h), sens.ctypes.data_as(C.POINTER(C.c_int32)), sens.shape[0],
                                          int(n_steps), int(checkpoint_every),
                                          C.byref(allocator) if allocator is not None else None, C.byref(out)))
    return out.value


def lbm_tape_destroy(t: int):
    if t:
        load_library().lbm_tape_destroy(C.c_void_p(t))


class Tape:
    """Recording of n_steps time steps of a Lattice (F32 or F64 storage) with
    the misfit of w at the sensor sites, and the transposed sweep that turns
    it into dL/dw*_e(t_n), dL/dw0 and dL/dwdot0 (include/lbm_adjoint.h).

    sensors: (ns, 2) integer (i, j) sites.  checkpoint_every: 0 keeps the
    misfits of every step, k > 0 keeps a state snapshot every k steps and
    recomputes each segment in the backward sweep."""

    def __init__(self, lattice: Lattice, sensors, n_steps: int, checkpoint_every: int = 0,
                 torch_allocator: bool = True):
        self.lattice = lattice
        self.torch = lattice.torch
        self.sensors = np.ascontiguousarray(np.asarray(sensors, dtype=np.int32).reshape(-1, 2))
        self.ns = self.sensors.shape[0]
        self.n_steps = int(n_steps)
        self._alloc = TorchAllocator(lattice.stream) if torch_allocator else None
        self.t = lbm_tape_create(lattice.h, self.sensors, self.n_steps, checkpoint_every,
                                 self._alloc.struct if self._alloc else None)

    def forward(self, targets, loss_to_host: bool = True):
        """Run n_steps steps of the lattice from its current state.  targets:
        (n_steps, ns) FP64 (numpy array or CUDA tensor).  Returns L (float)
        if loss_to_host, else None (no synchronisation)."""
        lib = load_library()
        torch = self.torch
        if isinstance(targets, torch.Tensor) and targets.is_cuda:
            tg = targets.to(torch.float64).contiguous()
            assert tg.numel() == self.n_steps * self.ns
            ptr, on_dev, keep = tg.data_ptr(), 1, tg
        else:
            keep = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(self.n_steps, self.ns))
            ptr, on_dev = keep.ctypes.data, 0
        loss = C.c_double(0.0)
        _check(lib.lbm_tape_forward(C.c_void_p(self.t), C.c_void_p(ptr), on_dev,
                                    C.byref(loss) if loss_to_host else None))
        del keep
        return loss.value if loss_to_host else None

    def backward(self, device: bool = True):
        """(dload (4, n_steps) FP64, dw0 (ny, nx), dwdot0 (ny, nx)) as CUDA
        tensors (enqueued on the lattice's stream) or, if not device, host
        numpy arrays."""
        lib = load_library()
        lat = self.lattice
        torch = self.torch
        if device:
            dload = torch.empty((4, self.n_steps), dtype=torch.float64, device="cuda")
            dw = torch.empty((lat.ny, lat.nx), dtype=lat.torch_dtype, device="cuda")
            dwd = torch.empty((lat.ny, lat.nx), dtype=lat.torch_dtype, device="cuda")
            ptrs = (dload.data_ptr(), dw.data_ptr(), dwd.data_ptr())
        else:
            dload = np.empty((4, self.n_steps))
            dw = np.empty((lat.ny, lat.nx), lat.np_dtype)
            dwd = np.empty((lat.ny, lat.nx), lat.np_dtype)
            ptrs = (dload.ctypes.data, dw.ctypes.data, dwd.ctypes.data)
        _check(lib.lbm_tape_backward(C.c_void_p(self.t), C.c_void_p(ptrs[0]), int(device), C.c_void_p(ptrs[1]),
                                     C.c_void_p(ptrs[2]), int(device), lat.dtype_code))
        return dload, dw, dwd

    def misfits(self) -> np.ndarray:
        """(n_steps, ns) misfits w^n(x_k) - target of the last recording."""
        out = np.empty((self.n_steps, self.ns))
        _check(load_library().lbm_tape_misfits(C.c_void_p(self.t), C.c_void_p(out.ctypes.data), 0))
        return out

    def close(self):
        if getattr(self, "t", None):
            lbm_tape_destroy(self.t)
            self.t = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lbm_adjoint(lattice: Lattice, sensors, n_steps: int, targets, checkpoint_every: int = 0,
                allocator: A.Allocator | None = None):
    """The one-call form of a tape's forward run and transposed sweep
    (lbm_adjoint): (L, dload (4, n_steps), dw0 (ny, nx), dwdot0 (ny, nx)) as
    host numpy arrays."""
    sens = np.ascontiguousarray(np.asarray(sensors, dtype=np.int32).reshape(-1, 2))
    tg = np.ascontiguousarray(np.asarray(targets, dtype=np.float64).reshape(int(n_steps), sens.shape[0]))
    loss = C.c_double(0.0)
    dload = np.empty((4, int(n_steps)))
    dw = np.empty((lattice.ny, lattice.nx), lattice.np_dtype)
    dwd = np.empty((lattice.ny, lattice.nx), lattice.np_dtype)
    _check(load_library().lbm_adjoint(C.c_void_p(lattice.h), sens.ctypes.data_as(C.POINTER(C.c_int32)),
                                      sens.shape[0], int(n_steps), int(checkpoint_every), C.c_void_p(tg.ctypes.data),
                                      0, C.byref(loss), C.c_void_p(dload.ctypes.data), 0, C.c_void_p(dw.ctypes.data),
                                      C.c_void_p(dwd.ctypes.data), 0, lattice.dtype_code,
                                      C.byref(allocator) if allocator is not None else None))
    return loss.value, dload, dw, dwd


def sensor_misfit(tape: Tape, edge: str, u, w0, wdot0, targets):
    """L = sum_{n,k} (w^n(x_k) - targets[n-1, k])^2 of tape.n_steps steps of
    the tape's lattice from step 0, with the loading of `edge` set to the
    series u (length n_steps) and initial fields (w0, wdot0), as a
    differentiable function of u, w0 and wdot0 (torch.autograd).  The
    gradient is that of the run with the cut schedule it took."""
    return _SensorMisfit.apply(u, w0, wdot0, tape, edge, targets)


def _autograd_function():
    import torch

    class SensorMisfitFn(torch.autograd.Function):
        @staticmethod
        def forward(ctx, u, w0, wdot0, tape, edge, targets):
            if u.numel() != tape.n_steps:
                raise ValueError("the load series must have one value per recorded step")
            lat = tape.lattice
            lat.reset()
            lat.set_loading(edge, "series", series=u)
            lat.set_fields(w0.detach(), wdot0.detach())
            loss = tape.forward(targets)
            ctx.tape = tape
            ctx.edge = A.EDGE_INDEX[edge]
            ctx.u_meta = (u.dtype, u.device)
            return torch.tensor(loss, dtype=torch.float64, device=w0.device)

        @staticmethod
        def backward(ctx, gL):
            dload, dw, dwd = ctx.tape.backward(device=True)
            gu = (gL * dload[ctx.edge]).to(ctx.u_meta[0]).to(ctx.u_meta[1])
            return gu, (gL * dw).to(dw.dtype), (gL * dwd).to(dwd.dtype), None, None, None

    return SensorMisfitFn


class _Lazy:
    fn = None

    def apply(self, *args):
        if _Lazy.fn is None:
            _Lazy.fn = _autograd_function()
        return _Lazy.fn.apply(*args)


_SensorMisfit = _Lazy()


# ----------------------------------------------------- row-slab decomposition

def lbm_decomp_plan(ny: int, jc: int, hh: int, n_ranks: int) -> list:
    """Row starts of lbm_decomp_plan's split (host only)."""
    out = (C.c_int32 * (n_ranks + 1))()
    _check(load_library().lbm_decomp_plan(int(ny), int(jc), int(hh), int(n_ranks), out))
    return list(out)


class SlabView:
    """Read-only view of one slab's handle (fields, crack state, masks)."""

    def __init__(self, h: int, problem: dict, storage: str, row0: int, rows: int):
        import torch
        self.torch = torch
        self.h = h
        self.problem = problem
        self.storage = storage
        self.row0, self.ny, self.nx = row0, rows, int(problem["nx"])
        self.np_dtype = np.float64 if storage == "f64" else np.float32

    fields = Lattice.fields
    cut_mask = Lattice.cut_mask
    crack_state = Lattice.crack_state
    history = Lattice.history
    crack_state_left = Lattice.crack_state_left
    history_left = Lattice.history_left
    dtype_code = Lattice.dtype_code


class Slab(Lattice):
    """Rows row0 .. row0 + rows - 1 of the lattice `problem` describes, as a
    lattice of its own (lbm_slab_create): one per process (or device).  Its
    halo rows come from the neighbouring slabs: after set_fields and after
    every step(1), call exchange(send_recv) -- or export_rows / import_rows
    with a transport of your own -- before anything else on the handle."""

    def __init__(self, problem: dict, row0: int, rows: int, storage: str = "f32", stream=None,
                 torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.problem = problem
        self.storage = storage
        self.row0, self.rows = int(row0), int(rows)
        self.nx, self.ny = int(problem["nx"]), self.rows
        self.global_ny = int(problem["ny"])
        self.np_dtype = np.float64 if storage == "f64" else np.float32
        self.torch_dtype = torch.float64 if storage == "f64" else torch.float32
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream_obj = stream
        self.stream = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
        g, lat, mat, cr, loads, keep = make_structs(problem, storage)
        self._alloc = TorchAllocator(self.stream) if torch_allocator else None
        self.line = False
        arr = (A.Loading * max(len(loads), 1))(*loads)
        out = C.c_void_p()
        _check(load_library().lbm_slab_create(C.byref(g), C.byref(lat), C.byref(mat), C.byref(cr) if cr.mode else None,
                                              arr if loads else None, len(loads), self.row0, self.rows,
                                              C.c_void_p(self.stream),
                                              C.byref(self._alloc.struct) if self._alloc else None, C.byref(out)))
        self.h = out.value
        periodic = problem.get("edges", ("free", "free", "dirichlet", "dirichlet"))[2] == "periodic"
        self.halo = (self.row0 > 0 or periodic, self.row0 + self.rows < self.global_ny or periodic)
        del keep

    def export_rows(self):
        """The slab's bottom and top rows of w (host arrays of nx values)."""
        out = []
        for side in (0, 1):
            a = np.empty(self.nx, self.np_dtype)
            _check(load_library().lbm_slab_export(C.c_void_p(self.h), side, C.c_void_p(a.ctypes.data), 0))
            out.append(a)
        return out

    def import_rows(self, below=None, above=None):
        """The neighbours' boundary rows into the halo rows (None: leave)."""
        for side, a in ((0, below), (1, above)):
            if a is None:
                continue
            a = np.ascontiguousarray(a, dtype=self.np_dtype)
            _check(load_library().lbm_slab_import(C.c_void_p(self.h), side, C.c_void_p(a.ctypes.data), 0))

    def set_fields(self, w=None, wdot=None):
        """This slab's rows of the lattice's fields (rows x nx arrays)."""
        Lattice.set_fields(self, w, wdot)


class Decomp:
    """A lattice split into row slabs on one GPU (include/lbm_decomp.h):
    one batched step launch and one halo-exchange launch per step, results
    bit-identical to the undivided Lattice."""

    def __init__(self, problem: dict, n_ranks: int, storage: str = "f32", row_start=None, stream=None,
                 torch_allocator: bool = True):
        import torch
        self.torch = torch
        self.problem = problem
        self.storage = storage
        self.nx, self.ny = int(problem["nx"]), int(problem["ny"])
        self.np_dtype = np.float64 if storage == "f64" else np.float32
        if stream is None:
            stream = torch.cuda.current_stream()
        self.stream = int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)
        g, lat, mat, cr, loads, keep = make_structs(problem, storage)
        self._alloc = TorchAllocator(self.stream) if torch_allocator else None
        arr = (A.Loading * max(len(loads), 1))(*loads)
        rs = None
        if row_start is not None:
            rs = (C.c_int32 * (n_ranks + 1))(*[int(x) for x in row_start])
        out = C.c_void_p()
        _check(load_library().lbm_decomp_create(C.byref(g), C.byref(lat), C.byref(mat), C.byref(cr) if cr.mode else None,
                                                arr if loads else None, len(loads), int(n_ranks), rs,
                                                C.c_void_p(self.stream),
                                                C.byref(self._alloc.struct) if self._alloc else None, C.byref(out)))
        self.d = out.value
        del keep

    @property
    def dtype_code(self) -> int:
        return A.STORAGE["f64"] if self.storage == "f64" else A.STORAGE["f32"]

    def step(self, n: int = 1):
        _check(load_library().lbm_decomp_step(C.c_void_p(self.d), int(n)))

    def set_fields(self, w=None, wdot=None):
        for which, arr in (("w", w), ("wdot", wdot)):
            if arr is None:
                continue
            a = np.ascontiguousarray(np.asarray(arr, dtype=self.np_dtype).reshape(self.ny, self.nx))
            _check(load_library().lbm_decomp_set_fields(C.c_void_p(self.d), A.FIELD[which], C.c_void_p(a.ctypes.data),
                                                        0, self.dtype_code))

    def fields(self):
        out = []
        for which in ("w", "wdot"):
            a = np.empty((self.ny, self.nx), self.np_dtype)
            _check(load_library().lbm_decomp_fields(C.c_void_p(self.d), A.FIELD[which], C.c_void_p(a.ctypes.data), 0,
                                                    self.dtype_code))
            out.append(a)
        return tuple(out)

    def info(self) -> dict:
        n, c = C.c_int32(), C.c_int32()
        _check(load_library().lbm_decomp_info(C.c_void_p(self.d), C.byref(n), C.byref(c)))
        return {"n_ranks": n.value, "crack_rank": c.value}

    def rank(self, r: int) -> SlabView:
        h, row0, rows = C.c_void_p(), C.c_int32(), C.c_int32()
        _check(load_library().lbm_decomp_rank(C.c_void_p(self.d), int(r), C.byref(h), C.byref(row0), C.byref(rows)))
        return SlabView(h.value, self.problem, self.storage, row0.value, rows.value)

    def close(self):
        if getattr(self, "d", None):
            load_library().lbm_decomp_destroy(C.c_void_p(self.d))
            self.d = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
