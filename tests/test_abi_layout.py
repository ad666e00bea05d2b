"""The ctypes mirrors of the C ABI structs have the header's size and field offsets: a small
C program built from include/rbe.h with gcc prints sizeof and offsetof of every field."""
import ctypes
import os
import shutil
import subprocess

import pytest

from paper_2110_14362_gb300 import _binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# status codes in the numbering of the library's specification (RBE_ESTATE = 6; RBE_ESAMPLE,
# which the specification does not list, after it), precisions, rho accumulations, samplers
ENUMS = ["RBE_OK", "RBE_EINVAL", "RBE_ENOMEM", "RBE_ECUDA", "RBE_ETIMEOUT", "RBE_ENONFINITE", "RBE_ESTATE",
         "RBE_ESAMPLE", "RBE_FP64", "RBE_FP32_PHASE", "RBE_RHO_FP64", "RBE_RHO_COMP32", "RBE_RHO_FP32",
         "RBE_SAMPLER_EXACT", "RBE_SAMPLER_OFFLINE", "RBE_SAMPLER_MH"]

STRUCTS = {
    "rbe_npt_params": B.NptParams,
    "rbe_system": B.System,
    "rbe_batch_item": B.BatchItem,
    "rbe_server_config": B.ServerConfig,
    "rbe_request": B.Request,
    "rbe_flex_params": B.FlexParams,
    "rbe_water_params": B.WaterParams,
    "rbe_flex_system": B.FlexSystem,
}


def _c_layout(tmp_path):
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rbe.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f in py._fields_:
            lines.append(f'printf("{cname} {f[0]} %zu\\n", offsetof({cname}, {f[0]}));')
    for name in ENUMS:
        lines.append(f'printf("{name} %d\\n", (int){name});')
    lines.append('printf("RBE_CELL_DOUBLES %d\\n", RBE_CELL_DOUBLES);')
    lines.append('printf("RBE_FLEX_CELL_DOUBLES %d\\n", RBE_FLEX_CELL_DOUBLES);')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    return {" ".join(l.split()[:-1]): int(l.split()[-1]) for l in out.splitlines()}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_ctypes_structs_match_header(tmp_path):
    c = _c_layout(tmp_path)
    for cname, py in STRUCTS.items():
        assert c[f"{cname} size"] == ctypes.sizeof(py), cname
        for f in py._fields_:
            assert c[f"{cname} {f[0]}"] == getattr(py, f[0]).offset, (cname, f[0])
    for name in ENUMS:
        assert c[name] == getattr(B, name), name
    assert (B.RBE_ESTATE, B.RBE_ESAMPLE) == (6, 7)
    assert c["RBE_CELL_DOUBLES"] == B.RBE_CELL_DOUBLES
    assert c["RBE_FLEX_CELL_DOUBLES"] == B.RBE_FLEX_CELL_DOUBLES
