"""The C-ABI library builds, loads and exports what include/*.h declare;
its struct layouts agree with the Python binding; argument validation
rejects bad configurations before touching a GPU.  No CUDA device needed."""
import ctypes as C
import os
import re
import subprocess

import pytest

from paper_2206_12412_gb300 import _abi as A
from paper_2206_12412_gb300 import build as B
from paper_2206_12412_gb300 import lbm

HEADERS = sorted(os.path.join(B.INCLUDE, f) for f in os.listdir(B.INCLUDE) if f.endswith(".h"))


@pytest.fixture(scope="module")
def lib():
    return lbm.load_library()


def declared_functions():
    names = set()
    for path in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(path).read(), flags=re.S)
        names |= set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text))
    return sorted(names)


def test_header_declares_core_calls():
    names = declared_functions()
    for core in ("lbm_create", "lbm_step", "lbm_fields", "lbm_crack_state", "lbm_destroy", "lbm_tape_create",
                 "lbm_tape_forward", "lbm_tape_backward"):
        assert core in names


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\sT\s(lbm_\w+)", out))
    for name in declared_functions():
        assert name in exported, name
        assert hasattr(lib, name)
        assert name in A.PROTOTYPES, name


def test_struct_layout_matches_header(tmp_path):
    structs = {"lbm_grid": A.Grid, "lbm_lattice": A.Lattice_, "lbm_material": A.Material, "lbm_crack": A.Crack,
               "lbm_crack_line": A.CrackLine, "lbm_loading": A.Loading, "lbm_allocator": A.Allocator, "lbm_crack_state_t": A.CrackStateT}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "lbm.h"', "int main(void){"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", B.INCLUDE, str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    got = {}
    for l in out:
        if l:
            c, f, v = l.split()
            got[(c, f)] = int(v)
    for cname, py in structs.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert got[(cname, fname)] == getattr(py, fname).offset, (cname, fname)


def _structs(**over):
    from paper_2206_12412_gb300 import workloads as W
    p = W.plain_fp64()
    p.update(over.pop("problem", {}))
    g, lat, mat, cr, loads, keep = lbm.make_structs(p, over.pop("storage", "f64"))
    for k, v in over.items():
        obj, field = k.split("__")
        setattr({"g": g, "lat": lat, "mat": mat, "cr": cr}[obj], field, v)
    return g, lat, mat, cr, loads, keep


@pytest.mark.parametrize("over,msg", [
    ({"g__nx": 0}, "nx"),
    ({"g__ny": 1}, "ny"),
    ({"g__dh": 0.0}, "dh"),
    ({"g__dt": float("nan")}, "dt"),
    ({"lat__omega": 0.8}, "omega"),
    ({"lat__storage": 7}, "storage"),
    ({"lat__velocity_set": 3}, "D2Q5"),
    ({"lat__velocity_set": 1, "lat__bc_mode": 0, "lat__storage": 2}, "D2Q9 needs"),
    ({"lat__velocity_set": 1, "lat__bc_mode": 0, "mat__mu": 0.8}, "3/4"),
    ({"lat__velocity_set": 0, "mat__mu": 0.6}, "1/2"),
    ({"mat__mu": 2.0}, "unstable"),
    ({"mat__rho": -1.0}, "rho"),
    ({"cr__y": 64.5}, "multiple of dh"),
    ({"cr__y": 2.0}, "too close"),
    ({"cr__x_tip": 128.0}, "left of"),
    ({"cr__x_tip": 126.6}, "narrow ligament"),
    ({"cr__x_start": 1.2}, "narrow ligament"),
    ({"lat__bc_mode": 3}, "boundary mode"),
    ({"lat__bc_mode": 2, "cr__x_start": 2.2}, "narrow ligament"),
    ({"lat__bc_mode": 2, "cr__x_tip": 125.6}, "narrow ligament"),
    ({"lat__bc_mode": 2, "cr__y": 3.0}, "too close"),
    ({"lat__bc_mode": 2, "cr__y": 125.0}, "too close"),
    ({"lat__bc_mode": 2, "g__nx": 3, "cr__mode": 0}, "nx >= 4"),
    ({"lat__bc_mode": 2, "g__ny": 3, "cr__mode": 0}, "ny >= 4"),
    ({"cr__x_start": 40.0}, "x_start"),
    ({"cr__mode": 9}, "crack mode"),
])
def test_create_rejects_bad_arguments(lib, over, msg):
    g, lat, mat, cr, loads, keep = _structs(**over)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create(g, lat, mat, cr, loads, 0, None)
    assert ei.value.status == A.LBM_ERR_ARG
    assert msg in str(ei.value)


def _line_structs(**over):
    from paper_2206_12412_gb300 import workloads as W
    p = W.with_line_crack(W.base_problem(40, 32, bc_mode="bounceback"), mode="prescribed", start=(6.3, 7.1),
                          tip=(14.2, 11.9), v_rel=0.6, r0=2.0)
    g, lat, mat, cr, loads, keep = lbm.make_structs(p, over.pop("storage", "f64"))
    for k, v in over.items():
        obj, field = k.split("__")
        setattr({"g": g, "lat": lat, "mat": mat, "cr": cr}[obj], field, v)
    return g, lat, mat, cr, loads, keep


@pytest.mark.parametrize("over,msg", [
    ({"cr__mode": 0}, "K-criterion mode"),
    ({"cr__mode": 5}, "K-criterion mode"),
    ({"lat__velocity_set": 1}, "D2Q5"),
    ({"lat__bc_mode": 2}, "link-local edges"),
    ({"lat__storage": 7}, "storage"),
    ({"cr__r0": 0.5}, "dh / 2"),
    ({"cr__r0": 0.0, "cr__r_min": 0.4}, "dh / 2"),
    ({"cr__x_start": -0.1}, "in the body"),
    ({"cr__y_tip": 32.5}, "in the body"),
    ({"cr__x_tip": 6.3, "cr__y_tip": 7.1}, "coincide"),
    ({"cr__x_start": 5.5, "cr__y_start": 5.5, "cr__x_tip": 9.5, "cr__y_tip": 9.5}, "site centre"),
    ({"cr__x_start": 5.5, "cr__y_start": 3.0, "cr__x_tip": 5.5, "cr__y_tip": 9.0}, "site centre"),
    ({"cr__v_rel": 1.0}, "v_rel"),
    ({"cr__mode": 3, "cr__K_C": 0.0}, "K_C"),
    ({"g__dh": 0.0}, "dh"),
    ({"cr__two_tips": 2}, "two_tips"),
    # the macroscopic rule: an edge crack's mouth, a crack one spacing from the bottom edge
    ({"lat__bc_mode": 1, "cr__x_start": 0.0, "cr__y_start": 16.3, "cr__x_tip": 8.0, "cr__y_tip": 19.1}, "outside the body"),
    ({"lat__bc_mode": 1, "cr__y_start": 1.2, "cr__y_tip": 5.9}, "outside the body"),
])
def test_create_line_rejects_bad_arguments(lib, over, msg):
    g, lat, mat, cr, loads, keep = _line_structs(**over)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_create_line(g, lat, mat, cr, loads, 0, None)
    assert ei.value.status == A.LBM_ERR_ARG
    assert msg in str(ei.value)


def test_create_line_accepts_macroscopic_faces_inside_the_body(lib):
    """The same crack inside the body passes every check with the macroscopic
    rule (without a GPU the call stops later, at the device query)."""
    g, lat, mat, cr, loads, keep = _line_structs(lat__bc_mode=1)
    try:
        h = lbm.lbm_create_line(g, lat, mat, cr, loads, 0, None)
    except lbm.LbmError as e:
        assert e.status != A.LBM_ERR_ARG, str(e)
    else:
        lbm.lbm_destroy(h)


def test_create_rejects_unpaired_periodic_and_bad_loads(lib):
    g, lat, mat, cr, loads, keep = _structs()
    g.edge[0] = A.EDGE["periodic"]
    with pytest.raises(lbm.LbmError, match="pairs"):
        lbm.lbm_create(g, lat, mat, cr, loads, 0, None)
    g, lat, mat, cr, loads, keep = _structs()
    loads[1].edge = loads[0].edge
    with pytest.raises(lbm.LbmError, match="repeated"):
        lbm.lbm_create(g, lat, mat, cr, loads, 0, None)
    g, lat, mat, cr, loads, keep = _structs()
    loads[0].kind = A.LOAD["series"]
    with pytest.raises(lbm.LbmError, match="series"):
        lbm.lbm_create(g, lat, mat, cr, loads, 0, None)


def test_null_handles_are_rejected(lib):
    assert lib.lbm_save(None, b"/tmp/x.lbm") == A.LBM_ERR_ARG
    assert lib.lbm_load(None, b"/tmp/x.lbm") == A.LBM_ERR_ARG
    assert lib.lbm_step(None, 1) == A.LBM_ERR_ARG
    assert lib.lbm_sync(None) == A.LBM_ERR_ARG
    assert lib.lbm_fields(None, 0, None, 0, 0) == A.LBM_ERR_ARG
    assert lib.lbm_crack_state(None, None, None, None, None, None, 0, None) == A.LBM_ERR_ARG
    assert lib.lbm_reset(None) == A.LBM_ERR_ARG
    assert lib.lbm_set_loading(None, None) == A.LBM_ERR_ARG
    out = C.c_void_p()
    assert lib.lbm_tape_create(None, None, 0, 1, 0, None, C.byref(out)) == A.LBM_ERR_ARG
    assert lib.lbm_tape_forward(None, None, 0, None) == A.LBM_ERR_ARG
    assert lib.lbm_tape_backward(None, None, 0, None, None, 0, 0) == A.LBM_ERR_ARG
    assert lib.lbm_tape_misfits(None, None, 0) == A.LBM_ERR_ARG
    lib.lbm_tape_destroy(None)
    lib.lbm_destroy(None)
    assert lbm.lbm_last_error() != ""
