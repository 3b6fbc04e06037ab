"""The ctypes structures of the binding have the C layout of include/cpm.h:
a small C program (gcc, no CUDA) prints sizeof and offsetof of every field,
and the ctypes sizes and offsets must equal them."""
import ctypes as C
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {
    "cpm_surface": ["kind", "param"],
    "oras_params": ["nparts", "overlap", "robin", "alpha", "alpha_cross", "store", "order", "coarse"],
    "oras_tuning": ["xplace", "lanes", "schedule", "ctas", "probe_timeout", "wait_polls"],
    "cpm_solve_params": ["restart", "maxit", "rtol", "mixed", "reorth", "inner_rtol", "timing"],
    "cpm_solve_info": ["iters", "restarts", "ir_steps", "rel_residual", "status", "ms_precond", "ms_operator",
                       "n_precond", "n_operator"],
    "cpm_schnakenberg": ["delta1", "delta2", "lambda", "Du", "Dv", "dt", "model"],
}
PY_NAME = {("cpm_schnakenberg", "lambda"): "lambda_"}


def c_layout():
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "cpm.h"', "int main(void) {"]
    for s, fields in STRUCTS.items():
        lines.append(f'  printf("{s} size %zu\\n", sizeof({s}));')
        for f in fields:
            lines.append(f'  printf("{s} {f} %zu\\n", offsetof({s}, {f}));')
    lines += ["  return 0;", "}"]
    with tempfile.TemporaryDirectory() as d:
        src, exe = os.path.join(d, "layout.c"), os.path.join(d, "layout")
        open(src, "w").write("\n".join(lines) + "\n")
        subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", exe, src], check=True)
        out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    res = {}
    for line in out.splitlines():
        parts = line.split()
        res[(parts[0], parts[1])] = int(parts[2])
    return res


def test_struct_layouts_match_the_header():
    from paper_2110_06322_gb300 import cpm
    lay = c_layout()
    for s, fields in STRUCTS.items():
        cls = getattr(cpm, s)
        assert C.sizeof(cls) == lay[(s, "size")], s
        for f in fields:
            assert getattr(cls, PY_NAME.get((s, f), f)).offset == lay[(s, f)], (s, f)
