"""The ctypes binding against the C header it marshals for (CPU): a small C
program, compiled with gcc against include/fwi.h, prints the size and field
offsets of every struct passed by pointer and the value of every enumerator;
the binding's ctypes structures and constants must agree with all of them.
A field added to a header struct without the binding (or the other way round)
fails here, before any GPU call could read a misplaced pointer."""

import ctypes
import json
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "fwi_model": ["physics", "nz", "nx", "dz", "dx", "order", "npml", "pml_R", "pml_vmax", "pml_f0", "vp", "vs",
                  "rho", "op"],
    "fwi_sources": ["nshots", "kind", "x0", "stf", "mt", "line_len"],
    "fwi_receivers": ["nrec", "iz", "ix"],
}
ENUMS = ["FWI_OK", "FWI_EINVAL", "FWI_ECFL", "FWI_ENOMEM", "FWI_ECUDA", "FWI_EUNSTABLE", "FWI_ETIMEOUT",
         "FWI_ENOTIMPL", "FWI_ACOUSTIC", "FWI_ELASTIC", "FWI_OP_DIVERGENCE", "FWI_OP_LAPLACIAN", "FWI_SRC_POINT",
         "FWI_SRC_GAUSSIAN", "FWI_SRC_MOMENT", "FWI_SRC_LINE"]


@pytest.fixture(scope="module")
def header_layout(tmp_path_factory):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    d = tmp_path_factory.mktemp("abi")
    lines = ["#include <stddef.h>", "#include <stdio.h>", '#include "fwi.h"', "int main(void) {", '  printf("{");']
    for s, fields in STRUCTS.items():
        lines.append(f'  printf("\\"{s}\\": {{\\"size\\": %zu", sizeof({s}));')
        for f in fields:
            lines.append(f'  printf(", \\"{f}\\": %zu", offsetof({s}, {f}));')
        lines.append('  printf("}, ");')
    lines.append('  printf("\\"enums\\": {");')
    for i, e in enumerate(ENUMS):
        lines.append(f'  printf("{", " if i else ""}\\"{e}\\": %d", (int){e});')
    lines += ['  printf("}}\\n");', "  return 0;", "}"]
    src = d / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = d / "layout"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe)], check=True)
    return json.loads(subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout)


@pytest.mark.parametrize("name", sorted(STRUCTS))
def test_ctypes_structs_match_the_header(header_layout, name):
    from paper_2003_06027_gb300 import fwi

    cls = {"fwi_model": fwi._Model, "fwi_sources": fwi._Sources, "fwi_receivers": fwi._Receivers}[name]
    want = header_layout[name]
    assert [f for f, _ in cls._fields_] == STRUCTS[name]
    assert ctypes.sizeof(cls) == want["size"]
    for f in STRUCTS[name]:
        assert getattr(cls, f).offset == want[f], f


def test_binding_constants_match_the_header(header_layout):
    from paper_2003_06027_gb300 import fwi

    e = header_layout["enums"]
    for k in ("FWI_ACOUSTIC", "FWI_ELASTIC", "FWI_OP_DIVERGENCE", "FWI_OP_LAPLACIAN", "FWI_SRC_POINT",
              "FWI_SRC_GAUSSIAN", "FWI_SRC_MOMENT", "FWI_SRC_LINE"):
        assert getattr(fwi, k) == e[k], k
    for code, name in fwi.STATUS.items():
        assert e[name] == code, name
    assert sorted(fwi.STATUS.values()) == sorted(k for k in e if k in ENUMS[:8])
