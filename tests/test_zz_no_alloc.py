"""sph_diagnostics_noalloc: the conservation sums without any device
allocation, for callers that cannot allocate (e.g. code running inside a CUDA
graph capture).  Checked through the C ABI against sph_diagnostics, the
context-based entry point, on two calls in a row (the static scratch is
shared and reused).  Kept in a file collected last."""
import ctypes as C

import numpy as np
import pytest

import sph_inputs

pytestmark = pytest.mark.gpu


def test_noalloc_diagnostics_matches_context_version():
    import torch

    import paper_2005_02656_gb300 as pkg
    pkg.build()
    from paper_2005_02656_gb300 import SphSim, _lib
    lib = _lib.load()
    s = sph_inputs.jittered_box(30, seed_index=77, vel_sigma=0.3)
    sim = SphSim(s)
    ref = sim.diagnostics()                       # existing entry point (context scratch)
    scale = np.array([np.abs(s["m"] * s[k]).sum() for k in ("vx", "vy", "vz")] +
                     [np.abs(0.5 * s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)).sum(),
                      np.abs(s["m"] * s["u"]).sum()] + [np.abs(s["m"]).sum() * 10.0] * 3)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for call in range(2):
        out = np.full(8, np.nan)
        rc = lib.sph_diagnostics_noalloc(C.byref(sim._st), out.ctypes.data_as(C.c_void_p), stream)
        assert rc == 0, (call, rc)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * scale.max())
        assert np.all(np.abs(out - ref) <= 1e-13 * scale), (call, out, ref)
    # a state larger than the static scratch is rejected
    big = _lib.SphState()
    big.n = 16_777_217
    for f in ("x", "y", "z", "vx", "vy", "vz", "m", "u"):
        setattr(big, f, sim.t["x"].data_ptr())
    out = np.zeros(8)
    assert lib.sph_diagnostics_noalloc(C.byref(big), out.ctypes.data_as(C.c_void_p), stream) == \
        _lib.SPH_ERR_INVALID_ARG
    sim.close()
