"""The oracle and the CUDA path share no code: neither imports or includes
the other, and only the seeded input module is common to both."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_2005_02656_gb300")
ORACLE = os.path.join(ROOT, "oracle")


def _files(top, exts):
    for d, _, names in os.walk(top):
        for n in names:
            if n.endswith(exts):
                yield os.path.join(d, n)


def test_product_path_does_not_use_the_oracle():
    for f in _files(PKG, (".py", ".cu", ".cuh", ".h", ".cpp")):
        text = open(f).read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, re.M), f
        assert "sph_oracle" not in text and "liboracle" not in text, f


def test_oracle_does_not_use_the_product_path():
    for f in _files(ORACLE, (".py", ".c", ".h")):
        text = open(f).read()
        assert "paper_2005_02656_gb300" not in text, f
        assert "libsph" not in text and "sph.h" not in text, f


def test_inputs_module_holds_no_method_arithmetic():
    text = open(os.path.join(ROOT, "sph_inputs", "__init__.py")).read()
    for word in ("kernel_norm", "sinc", "density", "iad", "momentum", "eos"):
        assert not re.search(rf"def \w*{word}", text, re.I), word
