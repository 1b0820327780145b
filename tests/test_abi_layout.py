"""The ctypes binding's structures match include/stencil.h field by field
(CPU, no GPU): a C program compiled against the header prints every field's
offset and every structure's size, and the binding's ctypes layouts must
agree.  A field added to a header structure but not to the binding (or in a
different order) shifts every later field the binding reads."""
import ctypes
import os
import shutil
import subprocess

import pytest

import paper_2310_16298_gb300 as sx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# C structure name -> the binding's ctypes class (fields in declaration order)
STRUCTS = {
    "stencil_options": sx.stencil_options,
    "stencil_plan_info_t": sx.stencil_plan_info_t,
    "stencil_batch_info_t": sx.stencil_batch_info_t,
    "stencil_request": sx.stencil_request,
    "stencil_request_stats": sx.stencil_request_stats,
    "stencil_server_stats_t": sx.stencil_server_stats_t,
}


def c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "stencil.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'    printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'    printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        name, key, value = line.split()
        layout[(name, key)] = int(value)
    return layout


def test_binding_structs_match_the_header(tmp_path):
    layout = c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert layout[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert layout[(name, field)] == getattr(cls, field).offset, (name, field)
