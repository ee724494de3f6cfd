"""The Python binding's ctypes structures against the C header: a small C
program compiled with the host compiler against include/egs.h prints every
public structure's size and field offsets, and each ctypes mirror must agree
field by field (a drift would silently corrupt every call that passes one)."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

from paper_1708_02835_gb300 import binding

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

STRUCTS = {
    "egs_info": binding.egs_info,
    "egs_opts": binding.egs_opts,
    "egs_trace_rec": binding.egs_trace_rec,
    "egs_serve_config": binding.egs_serve_config,
    "egs_serve_stats_t": binding.egs_serve_stats,
}


def _c_layout(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no host C compiler")
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "egs.h"', "int main(void) {"]
    for cname, cls in STRUCTS.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for fname, _ in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, fname, cname, fname))
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True,
                   capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    layout = {}
    for line in out.splitlines():
        a, b, v = line.split()
        layout[(a, b)] = int(v)
    return layout


def test_ctypes_mirrors_match_the_header(tmp_path):
    layout = _c_layout(tmp_path)
    for cname, cls in STRUCTS.items():
        assert ctypes.sizeof(cls) == layout[(cname, "size")], cname
        for fname, _ in cls._fields_:
            assert getattr(cls, fname).offset == layout[(cname, fname)], (cname, fname)


def test_enums_match_the_header():
    text = open(os.path.join(ROOT, "include", "egs.h")).read()
    for name in ("EGS_OK", "EGS_ERR_ARG", "EGS_ERR_NOT_PD", "EGS_ERR_OOM", "EGS_ERR_CUDA", "EGS_ERR_TIMEOUT",
                 "EGS_ERR_BUSY", "EGS_ERR_UNIMPLEMENTED", "EGS_ERR_INACCURATE", "EGS_FP64", "EGS_MIX_FP32",
                 "EGS_MIX_TF32", "EGS_MIX_BF16"):
        m = re.search(r"\b%s\s*=\s*(\d+)" % name, text)
        assert m, name
        assert int(m.group(1)) == getattr(binding, name), name
    assert binding.PRECISIONS == {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
    assert len(binding.TRACE_CLASSES) == 7
