"""The Python binding agrees with the C header on the CPU: the layout of the
two structs the binding passes by pointer (sizes and field offsets as a C
compiler lays them out from include/vplbm.h) and the value of every enum
constant the header declares."""
import ctypes as C
import os
import re
import shutil
import subprocess

import pytest

from paper_2110_00967_gb300 import vplbm as V

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vplbm.h")

STRUCTS = {"vplbm_config": V.vplbm_config, "vplbm_body": V.vplbm_body}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vplbm.h"', "int main(void) {"]
    for name, cls in STRUCTS.items():
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'  printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c99", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {tuple(l.split()[:2]): int(l.split()[2]) for l in out.splitlines()}


def test_struct_layout_matches_the_header(tmp_path):
    got = _c_layout(tmp_path)
    for name, cls in STRUCTS.items():
        assert got[(name, "size")] == C.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


def test_enum_constants_match_the_header():
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    consts = dict((k, int(v)) for k, v in re.findall(r"\bVPLBM_([A-Z0-9_]+)\s*=\s*(\d+)", text))
    assert len(consts) >= 25
    checked = 0
    for k, v in consts.items():
        if hasattr(V, k):
            assert getattr(V, k) == v, k
            checked += 1
    # every constant the binding exposes under the header's name is checked;
    # these are the ones the tests and the bench rely on
    for k in ("OK", "EINVAL", "ESTATE", "F64", "F32", "F16_OFS", "BF16_OFS", "TRT", "PERIODIC",
              "INLET_BB", "OUTLET_CONVECTIVE", "OUTLET_FREE", "NOSLIP_BB", "SYMMETRY",
              "MEM", "SIM", "ANGOT"):
        assert hasattr(V, k) and getattr(V, k) == consts[k], k
    assert checked >= 17
