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
    assert p.pair_mode == 0      # SPH_PAIRS_STAGED
    assert p.energy_dt == 0.0 and p.angular_sums == 0
    assert abs(p.gamma - 5.0 / 3.0) < 1e-15 and p.alpha == 1.0 and p.courant == 0.2
    src = tmp_path / "layout.c"
    src.write_text(
        '#include <stdio.h>\n#include <stddef.h>\n#include "sph.h"\n'
        'int main(void){printf("%zu %zu %zu %zu %zu %zu %zu\\n", sizeof(sph_state), sizeof(sph_params),'
        ' offsetof(sph_state, n), offsetof(sph_params, sinc_n), offsetof(sph_params, gradh),'
        ' offsetof(sph_params, pair_mode), offsetof(sph_params, angular_sums));'
        'return 0;}\n')
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    vals = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                           check=True).stdout.split()]
    assert vals == [C.sizeof(SphState), C.sizeof(SphParams), SphState.n.offset,
                    SphParams.sinc_n.offset, SphParams.gradh.offset, SphParams.pair_mode.offset,
                    SphParams.angular_sums.offset]


def test_null_arguments_are_rejected(lib):
    # host-side argument checks only: no device work is enqueued
    assert lib.sph_init(None, 10, None) == -1
    assert lib.sph_step(None, None, None, None) == -1
    assert lib.sph_error_word(None, None) == -1
    assert lib.sph_last_error(None) == b"no context"


def _params(lib, **kw):
    from paper_2005_02656_gb300._lib import SphParams
    p = SphParams()
    lib.sph_default_params(C.byref(p))
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("field,value", [
    ("gamma", 1.0), ("alpha", -0.1), ("courant", 0.0), ("dt_growth", 0.9), ("ng_target", -1),
    ("max_nb", 0), ("max_nb", 162), ("max_nb", 4100), ("sinc_n", 0.5), ("sinc_n", 6.5),
    ("sinc_n", 13.0), ("precision", 7), ("kernel_mode", 3), ("gradh", 2), ("pair_mode", 2),
    ("energy_dt", -1.0), ("angular_sums", 2)])
def test_invalid_params_are_rejected_before_any_device_work(lib, field, value):
    # sph_init validates its parameters on the host and returns before any
    # CUDA call, so this runs without a GPU
    from paper_2005_02656_gb300._lib import SPH_ERR_INVALID_ARG
    p = _params(lib, **{field: value})
    ctx = C.c_void_p(1)
    assert lib.sph_init(C.byref(p), 1000, C.byref(ctx)) == SPH_ERR_INVALID_ARG
    assert not ctx.value


def test_param_combinations_and_sizes_are_rejected(lib):
    from paper_2005_02656_gb300._lib import SPH_ERR_INVALID_ARG, SPH_KERNEL_TABLE
    ctx = C.c_void_p()
    p = _params(lib, gradh=1, kernel_mode=SPH_KERNEL_TABLE)     # grad-h needs the exact kernel
    assert lib.sph_init(C.byref(p), 1000, C.byref(ctx)) == SPH_ERR_INVALID_ARG
    p = _params(lib)
    p.periodic[1] = 1
    p.box_lo[1], p.box_hi[1] = 1.0, 1.0                          # periodic axis of zero length
    assert lib.sph_init(C.byref(p), 1000, C.byref(ctx)) == SPH_ERR_INVALID_ARG
    p = _params(lib)
    for n_max in (0, -5, (1 << 27) + 1):                         # list entries hold 27-bit indices
        assert lib.sph_init(C.byref(p), n_max, C.byref(ctx)) == SPH_ERR_INVALID_ARG
    assert not ctx.value


def test_ensemble_defaults_and_host_checks(lib):
    from paper_2005_02656_gb300._lib import EnsConfig, SPH_ERR_INVALID_ARG, SPH_FP32_MIXED
    c = EnsConfig()
    lib.sph_ens_default_config(C.byref(c))
    assert (c.cell_factor, c.blocks_per_sm, c.test_skip_block, c.find_window,
            c.threads_per_particle, c.momentum_threads) == (1.0, 0, -1, 512, 1, 4)
    p = _params(lib, precision=SPH_FP32_MIXED)
    n = (C.c_int64 * 1)(100)
    d3 = (C.c_double * 3)(0, 0, 0)
    i3 = (C.c_int * 3)(1, 1, 1)
    a1 = (C.c_double * 1)(1.0)
    e = C.c_void_p()
    assert lib.sph_ensemble_init(C.byref(p), 0, n, d3, d3, i3, a1, C.byref(e)) == SPH_ERR_INVALID_ARG
    p64 = _params(lib)                                           # the ensemble is FP32-mixed only
    assert lib.sph_ensemble_init(C.byref(p64), 1, n, d3, d3, i3, a1, C.byref(e)) == SPH_ERR_INVALID_ARG
    assert not e.value


def test_missing_library_fails_loudly(tmp_path):
    """No CPU fallback: without libsph.so the binding raises."""
    from paper_2005_02656_gb300 import _lib
    saved = _lib._lib
    _lib._lib = None
    try:
        with pytest.raises(RuntimeError, match="no fallback"):
            _lib.load(str(tmp_path / "libsph.so"))
    finally:
        _lib._lib = saved
