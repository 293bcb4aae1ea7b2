"""The Python binding's ctypes structures match the C header field by field.

A small C program is compiled against include/sptrsv.h with the host compiler;
it prints sizeof and every field's offsetof, which must equal what ctypes lays
out for the binding's structures (a missing or reordered field in either would
silently corrupt every call that passes the struct)."""
import os
import shutil
import subprocess

import pytest

import paper_2503_05408_gb300 as sp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    ("sptrsv_csr", sp.CSRStruct),
    ("sptrsv_analyze_opts", sp.AnalyzeOpts),
    ("sptrsv_stats", sp.Stats),
    ("sptrsv_solve_opts", sp.SolveOpts),
    ("sptrsv_report", sp.Report),
    ("sptrsv_serve_opts", sp.ServeOpts),
    ("sptrsv_serve_statistics", sp.ServeStats),
]


def test_ctypes_layout_matches_header(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "sptrsv.h"', "int main(void) {"]
    for cname, py in PAIRS:
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            a, b, v = ln.split()
            got[(a, b)] = int(v)
    for cname, py in PAIRS:
        assert got[(cname, "size")] == ctypes_sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def ctypes_sizeof(t):
    import ctypes
    return ctypes.sizeof(t)
