"""The binding's mirrors of the C ABI's structs have the header's layout.

A C program compiled against include/geo3d.h prints the size of every
struct the binding mirrors and the offset of each of its fields; the ctypes
structures (and the numpy record type of a query) must agree byte for byte,
so a field added to the header without the binding (or the other way round)
fails here, on the CPU, before any call passes a misread struct."""
import ctypes as C
import os
import shutil
import subprocess

import pytest

from paper_1808_09571_gb300 import geo3d

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
MIRRORS = {"g3d_config": geo3d.g3d_config, "g3d_query": geo3d.g3d_query, "g3d_stats": geo3d.g3d_stats,
           "g3d_kernel_time": geo3d.g3d_kernel_time}


def _c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "geo3d.h"', "int main(void) {"]
    for sname, cls in MIRRORS.items():
        lines.append(f'  printf("{sname} . %zu\\n", sizeof({sname}));')
        for fname, _ in cls._fields_:
            lines.append(f'  printf("{sname} {fname} %zu\\n", offsetof({sname}, {fname}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([gcc, "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        s, f, v = line.split()
        layout[(s, f)] = int(v)
    return layout


def test_ctypes_mirrors_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for sname, cls in MIRRORS.items():
        assert C.sizeof(cls) == layout[(sname, ".")], sname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == layout[(sname, fname)], (sname, fname)


def test_query_records_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    dt = geo3d.Context.QUERY_DTYPE
    assert dt.itemsize == layout[("g3d_query", ".")]
    for fname in dt.names:
        assert dt.fields[fname][1] == layout[("g3d_query", fname)], fname
