"""The Python binding's ctypes structures must lay out exactly like the C
structs of include/hsga.h: a plain C program built with gcc against the
header prints every field's offset and every struct's size, and the binding's
structures must agree field by field (no GPU, no CUDA)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_2404_10861_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = [binding.hsga_config, binding.hsga_stats, binding.hsga_batch_run_info,
           binding.hsga_batch_stats]


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "hsga.h"', "int main(void) {"]
    for st in STRUCTS:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in st._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    d = tmp_path_factory.mktemp("abi")
    src, exe = d / "layout.c", d / "layout"
    src.write_text("\n".join(lines) + "\n")
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        parts = line.split()
        layout[tuple(parts[:-1])] = int(parts[-1])
    return layout


@pytest.mark.parametrize("st", STRUCTS, ids=lambda s: s.__name__)
def test_ctypes_structs_match_the_header(c_layout, st):
    name = st.__name__
    assert ctypes.sizeof(st) == c_layout[(name, "size")]
    for field, _ in st._fields_:
        assert getattr(st, field).offset == c_layout[(name, field)], field
    # and the header declares no field the binding does not know (one that
    # trailing padding would hide from the size check)
    assert header_fields(name) == [f for f, _ in st._fields_]


def header_fields(name):
    """Member names of `typedef struct name {...} name;` in include/hsga.h."""
    text = open(os.path.join(ROOT, "include", "hsga.h")).read()
    body = text[text.index(f"typedef struct {name} {{"):]
    body = body[body.index("{") + 1:body.index(f"}} {name};")]
    body = re.sub(r"/\*.*?\*/", " ", body, flags=re.S)
    body = re.sub(r"//[^\n]*", " ", body)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [v.strip() for v in decl.split(None, 1)[1].split(",")]
    return names
