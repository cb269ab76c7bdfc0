"""The C ABI (include/sph.h) without a GPU: the library builds, loads, exports
every declared entry point, and the ctypes structures match the C layout."""
import ctypes as C
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sph.h")


@pytest.fixture(scope="module")
def lib():
    import paper_2005_02656_gb300 as pkg
    pkg.build()
    from paper_2005_02656_gb300 import _lib
    return _lib.load()


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"SPH_API\s+[\w\s\*]+?\b(sph_\w+)\s*\(", txt)))


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert len(names) >= 17
    for n in names:
        assert hasattr(lib, n), n
    from paper_2005_02656_gb300 import _lib
    assert sorted(_lib.EXPORTS) == names


def test_default_params_and_layout(lib, tmp_path):
    from paper_2005_02656_gb300._lib import SphParams, SphState
    p = SphParams()
    lib.sph_default_params(C.byref(p))
    assert p.max_nb == 160 and p.ng_target == 100 and p.sinc_n == 6.0
    assert abs(p.gamma - 5.0 / 3.0) < 1e-15 and p.alpha == 1.0 and p.courant == 0.2
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sph.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu\\n", sizeof(sph_state), sizeof(sph_params),'
        ' offsetof(sph_state, n), offsetof(sph_params, sinc_n), offsetof(sph_params, gradh));'
        'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [C.sizeof(SphState), C.sizeof(SphParams), SphState.n.offset,
                    SphParams.sinc_n.offset, SphParams.gradh.offset]


def test_null_arguments_are_rejected(lib):
    # host-side argument checks only: no device work is enqueued
    assert lib.sph_init(None, 10, None) == -1
    assert lib.sph_step(None, None, None, None) == -1
    assert lib.sph_error_word(None, None) == -1
    assert lib.sph_last_error(None) == b"no context"
