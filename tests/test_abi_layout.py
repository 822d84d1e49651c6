"""The ctypes structures of the binding have the layout of the C structures in
include/dualip.h: a plain C program built from the header with gcc prints
sizeof and offsetof of every field, and the binding must agree field by
field (no GPU or CUDA toolkit needed)."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2603_04621_gb300 as d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C struct name -> binding class; field names are the same on both sides
STRUCTS = {
    "dualip_problem_desc": d.ProblemDesc,
    "dualip_eval": d.Eval,
    "dualip_solve_opts": d.SolveOpts,
    "dualip_solve_result": d.SolveResult,
    "dualip_autotune_result": d.AutotuneResult,
    "dualip_server_opts": d.ServerOpts,
    "dualip_request_info": d.RequestInfo,
    "dualip_server_stats": d.ServerStats,
}


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "dualip.h"',
             "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append(f'  printf("{cname} . %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["  return 0;", "}"]
    tmp = tmp_path_factory.mktemp("abi")
    src = tmp / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    table = {}
    for ln in out.splitlines():
        cname, fname, v = ln.split()
        table[(cname, fname)] = int(v)
    return table


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_binding_structs_match_the_header(c_layout, cname):
    cls = STRUCTS[cname]
    assert ctypes.sizeof(cls) == c_layout[(cname, ".")], "size"
    for fname, _ in cls._fields_:
        assert getattr(cls, fname).offset == c_layout[(cname, fname)], fname
