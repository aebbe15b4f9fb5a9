"""The binding's ctypes structs against the C header (no GPU).

A C program built from include/gwstream.h prints sizeof of each descriptor
and statistics struct and offsetof of every field the binding declares; the
binding's ctypes layout must agree field by field, so a field added to one
side only (or in another order) fails here instead of corrupting a call.
"""
import os
import shutil
import subprocess

import pytest

from paper_2108_12430_gb300 import gwstream as G

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [G.gw_model_desc, G.gw_stream_desc, G.gw_server_desc, G.gw_server_stats, G.gw_trainer_desc]


def c_layout(tmp_path):
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "gwstream.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} sizeof %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([gcc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    res = {}
    for ln in out.splitlines():
        name, key, val = ln.split()
        res[(name, key)] = int(val)
    return res


def test_ctypes_structs_match_the_header(tmp_path):
    c = c_layout(tmp_path)
    for st in STRUCTS:
        name = st.__name__
        assert c[(name, "sizeof")] == G.C.sizeof(st), name
        for field, _ in st._fields_:
            assert c[(name, field)] == getattr(st, field).offset, (name, field)
