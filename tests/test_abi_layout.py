"""The binding's ctypes mirrors of the C ABI's structures have the layout the C compiler
gives include/ddlra.h: every structure's size and every field's offset, from a small C
program compiled against the header (CPU only)."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_2602_14854_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"dd_grid": binding.Grid, "dd_tiling": binding.Tiling,
           "dd_quadrature": binding.Quadrature, "dd_fields": binding.Fields,
           "dd_options": binding.Options, "dd_allocator": binding.Allocator}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "ddlra.h"', 'int main(void) {']
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} sizeof %zu\\n", sizeof({cname}));')
        for fname, _ in py._fields_:
            lines.append(f'  printf("{cname} {fname} %zu\\n", offsetof({cname}, {fname}));')
    lines += ['  return 0;', '}']
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c99", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_ctypes_structures_match_the_header(tmp_path):
    lay = c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert lay[(cname, "sizeof")] == C.sizeof(py), cname
        for fname, _ in py._fields_:
            assert lay[(cname, fname)] == getattr(py, fname).offset, (cname, fname)
