"""The binding's ctypes structures against the C layout of include/ewos.h.

A small C program, compiled with the host compiler against the header, prints sizeof of every
structure of the ABI and offsetof of every field the binding declares (by the binding's field
names, so a renamed, missing or reordered field fails to compile or to match).  No GPU needed.
"""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2608_07017_b300 import ewos

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PAIRS = [
    (ewos._Domain, "ewos_domain"),
    (ewos.BuildOpts, "ewos_build_opts"),
    (ewos.BuildReport, "ewos_build_report"),
    (ewos._Problem, "ewos_problem"),
    (ewos.SolveReport, "ewos_solve_report"),
    (ewos.AdamOpts, "ewos_adam_opts"),
    (ewos.AdamReport, "ewos_adam_report"),
    (ewos.ServerOpts, "ewos_server_opts"),
    (ewos.ServerStats, "ewos_server_stats"),
    (ewos.RequestTiming, "ewos_request_timing"),
]


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs a host C compiler")
def test_ctypes_structures_match_the_header(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ewos.h"', "int main(void) {"]
    for cls, cname in PAIRS:
        lines.append(f'    printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            lines.append(f'    printf("{cname}.{fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    c = dict(line.rsplit(" ", 1) for line in out.strip().splitlines())
    for cls, cname in PAIRS:
        assert int(c[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(c[f"{cname}.{fname}"]) == getattr(cls, fname).offset, f"{cname}.{fname}"
