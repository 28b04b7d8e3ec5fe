"""The C-ABI library builds, loads and exports every symbol include/fdst.h
declares; host-side argument validation (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "fdst.h")


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(fdst_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    import paper_1712_00403_gb300 as pkg
    from paper_1712_00403_gb300 import build
    if not os.path.exists(pkg.LIB_PATH):
        build.build()
    return pkg.load_library()


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["fdst_setup", "fdst_destroy", "fdst_apply_prec", "fdst_matvec", "fdst_solve", "fdst_last_error"]:
        assert n in names


def test_every_declared_symbol_is_exported(lib):
    import paper_1712_00403_gb300 as pkg
    out = subprocess.run(["nm", "-D", "--defined-only", pkg.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fdst_[a-z_0-9]+)", out))
    for n in _declared():
        assert n in exported, n
        assert hasattr(lib, n)
    assert set(pkg.ENTRY_POINTS) <= exported
    # every declared entry point is bound, with its argument types (ctypes cannot convert
    # a Python float without them)
    assert set(_declared()) <= set(pkg.ENTRY_POINTS)
    for n in pkg.ENTRY_POINTS:
        assert getattr(lib, n).argtypes is not None, n


def _desc(pkg, knots, p, dim=None, **kw):
    d = pkg.Desc()
    d.dim = dim if dim is not None else len(knots)
    d.degree = p
    keep = [np.ascontiguousarray(k, dtype=np.float64) for k in knots]
    for e, k in enumerate(keep):
        d.h_knots[e] = k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        d.nknots[e] = len(k)
    d.viscosity = 1.0
    d.max_rhs = kw.get("max_rhs", 1)
    d.fd_precision = kw.get("fd_precision", 0)
    d.geometry = kw.get("geometry", 0)
    d.variant = kw.get("variant", 0)
    d._keep = keep
    return d


@pytest.mark.parametrize("knots,p,why", [
    ([[0, 0, 0.5, 1, 1]] * 2, 2, "not open"),
    ([[0, 0, 0, 0.6, 0.4, 1, 1, 1]] * 2, 2, "nondecreasing"),
    ([[0, 0, 0, 0.5, 0.5, 0.5, 1, 1, 1]] * 2, 2, "multiplicity"),
    ([[0, 0, 0, 1, 1, 1]] * 2, 0, "degree"),
])
def test_invalid_knots_rejected_on_host(lib, knots, p, why):
    import paper_1712_00403_gb300 as pkg
    d = _desc(pkg, knots, p)
    h = ctypes.c_void_p()
    code = lib.fdst_setup(ctypes.byref(d), ctypes.byref(h))
    assert code == 1, why          # FDST_INVALID_ARGUMENT
    assert h.value is None
    assert len(lib.fdst_last_error()) > 0


def test_bad_dim_and_null_arguments(lib):
    import paper_1712_00403_gb300 as pkg
    d = _desc(pkg, [[0, 0, 0, 1, 1, 1]] * 2, 2, dim=4)
    h = ctypes.c_void_p()
    assert lib.fdst_setup(ctypes.byref(d), ctypes.byref(h)) == 1
    assert lib.fdst_setup(None, ctypes.byref(h)) == 1
    assert lib.fdst_apply_prec(None, None, None, 1, None) == 1
    assert lib.fdst_destroy(None) == 0


def test_new_entry_points_validate_on_the_host(lib):
    """Argument checks that return before any device work: the block preconditioner,
    GMRES, the conversions and the kernel timing reject NULL handles and bad codes."""
    import paper_1712_00403_gb300 as pkg
    info = (pkg.SolveInfo * 1)()
    vp = ctypes.c_void_p
    assert lib.fdst_apply_block_prec(None, pkg.PREC_PT, vp(1), vp(2), 1, None) == 1
    assert lib.fdst_solve_gmres(None, pkg.PREC_PT, pkg.GMRES_AUTO, vp(1), vp(2), 1, 1e-8, 10, 10, info, None) == 1
    assert lib.fdst_convert(7, vp(1), vp(2), 4, None) == 1          # unknown kind
    assert lib.fdst_convert(0, None, vp(2), 4, None) == 1           # NULL input with n > 0
    assert lib.fdst_convert(0, None, None, 0, None) == 0            # nothing to do
    assert lib.fdst_get_kernel_timing(None, None, None) == 1
    assert lib.fdst_check_bounded_wait(None, None) == 1
    assert "NULL" in lib.fdst_last_error().decode()


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes mirrors of fdst_desc, fdst_sizes, fdst_solve_info and
    fdst_server_opts have the header's sizes and field offsets (a C program compiled
    against include/fdst.h prints them)."""
    import shutil

    import paper_1712_00403_gb300 as pkg
    if shutil.which("gcc") is None:
        pytest.skip("gcc is not available")
    mirrors = {"fdst_desc": pkg.Desc, "fdst_sizes": pkg.Sizes, "fdst_solve_info": pkg.SolveInfo,
               "fdst_server_opts": pkg.ServerOpts}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fdst.h"', "int main(void) {"]
    for c, py in mirrors.items():
        lines.append(f'  printf("{c} size %zu\\n", sizeof({c}));')
        for name, _ in py._fields_:
            lines.append(f'  printf("{c} {name} %zu\\n", offsetof({c}, {name}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(ln.split()[:2]): int(ln.split()[2]) for ln in out if ln}
    for c, py in mirrors.items():
        assert got[(c, "size")] == ctypes.sizeof(py), c
        for name, _ in py._fields_:
            assert got[(c, name)] == getattr(py, name).offset, (c, name)


def test_struct_members_match_the_header():
    """Same member names in the same order as the header declares them (an extra
    trailing int could hide in padding from the size check)."""
    import paper_1712_00403_gb300 as pkg
    text = open(HEADER).read()
    mirrors = {"fdst_desc": pkg.Desc, "fdst_sizes": pkg.Sizes, "fdst_solve_info": pkg.SolveInfo,
               "fdst_server_opts": pkg.ServerOpts}
    for c, py in mirrors.items():
        body = re.search(r"typedef struct \{((?:(?!typedef struct).)*?)\}\s*" + c + r"\s*;", text, re.S).group(1)
        body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
        names = re.findall(r"\**\s*([A-Za-z_][A-Za-z_0-9]*)\s*(?:\[[^\]]*\])*\s*;", body)
        assert names == [n for n, _ in py._fields_], (c, names)
