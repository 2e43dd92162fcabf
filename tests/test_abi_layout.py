"""The binding's ctypes structures match include/askit.h field for field:
a C program compiled by gcc against the header prints every field's offset
and each structure's size, and the ctypes mirrors must agree (CPU only)."""
import ctypes
import json
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
STRUCTS = {"askit_params": "Params", "askit_info": "Info", "askit_tune_entry": "TuneEntry"}


def header_fields():
    """Field names of each typedef'd struct of the header, in order."""
    src = open(os.path.join(ROOT, "include", "askit.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for body, name in re.findall(r"typedef struct \{(.*?)\}\s*(askit_[a-z_]+);", src, flags=re.S):
        fields = []
        for decl in body.split(";"):
            decl = decl.strip()
            if not decl:
                continue
            names = decl.split(None, 1)[1]
            for n in names.split(","):
                fields.append(re.sub(r"\[.*\]", "", n).strip())
        out[name] = fields
    return out


@pytest.fixture(scope="module")
def c_layout(tmp_path_factory):
    fields = header_fields()
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "askit.h"', "int main(void) {", 'printf("{");']
    first = True
    for s, fs in fields.items():
        for f in fs + ["__size__"]:
            expr = f"sizeof({s})" if f == "__size__" else f"offsetof({s}, {f})"
            lines.append(f'printf("{"" if first else ","}\\"{s}.{f}\\": %zu", (size_t)({expr}));')
            first = False
    lines += ['printf("}\\n");', "return 0; }"]
    d = tmp_path_factory.mktemp("abi")
    c, exe = d / "layout.c", d / "layout"
    c.write_text("\n".join(lines))
    subprocess.check_call(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    return json.loads(subprocess.check_output([str(exe)]).decode())


def test_every_header_struct_is_mirrored():
    assert set(header_fields()) == set(STRUCTS)


@pytest.mark.parametrize("cname", sorted(STRUCTS))
def test_ctypes_mirror_matches_the_header(cname, c_layout):
    from paper_1410_0260_gb300 import askit
    py = getattr(askit, STRUCTS[cname])
    names = [f for f, _ in py._fields_]
    assert names == header_fields()[cname]
    for f in names:
        assert getattr(py, f).offset == c_layout[f"{cname}.{f}"], f
    assert ctypes.sizeof(py) == c_layout[f"{cname}.__size__"]
