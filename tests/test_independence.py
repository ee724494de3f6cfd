"""The oracle and the CUDA path share no code and neither uses the other, and
the product has no CPU fallback: without its library the binding raises."""
import os
import re
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PRODUCT = os.path.join(ROOT, "paper_1708_02835_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _sources(top, exts):
    for d, _, files in os.walk(top):
        if "_build" in d or "__pycache__" in d:
            continue
        for f in files:
            if f.endswith(exts):
                yield os.path.join(d, f)


def test_product_never_refers_to_the_oracle():
    for path in _sources(PRODUCT, (".py", ".cu", ".cuh", ".h", ".c")):
        text = open(path).read()
        assert not re.search(r"\boracle\b", text), path
    for path in (os.path.join(ROOT, "include", "egs.h"),):
        assert "oracle" not in open(path).read()


def test_oracle_never_refers_to_the_product():
    for path in _sources(ORACLE, (".py", ".c", ".h")):
        text = open(path).read()
        assert "egs.h" not in text and "paper_1708_02835_gb300" not in text and "csrc" not in text, path


def test_missing_library_raises_instead_of_falling_back(tmp_path):
    code = (
        "import paper_1708_02835_gb300.build as b\n"
        "b.LIB = %r\n"
        "from paper_1708_02835_gb300 import binding\n"
        "try:\n"
        "    binding.load_library(build_if_missing=False)\n"
        "except RuntimeError as e:\n"
        "    print('raised', 'not built' in str(e))\n"
        "else:\n"
        "    print('loaded')\n" % str(tmp_path / "missing" / "libegs.so"))
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=120)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr
