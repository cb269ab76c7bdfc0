"""sph_diagnostics_noalloc: the conservation sums without any device
allocation, for callers that cannot allocate device memory (a host that owns
all device memory through its own pool, or code that holds no context).
Checked through the C ABI against sph_diagnostics, the context-based entry
point, on two calls in a row (the static scratch is shared and reused), at
the largest accepted size followed by a small call, and on a stream under
graph capture, which it must refuse without breaking the capture.  Kept in a
file collected last."""
import ctypes as C

import numpy as np
import pytest

import sph_inputs

pytestmark = pytest.mark.gpu

N_MAX = 16_777_216      # 8192 blocks x 2048 particles: the whole static array


def _lib():
    import paper_2005_02656_gb300 as pkg
    pkg.build()
    from paper_2005_02656_gb300 import _lib as L
    return L, L.load()


def _stream():
    import torch
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _scale(s):
    return np.array([np.abs(s["m"] * s[k]).sum() for k in ("vx", "vy", "vz")] +
                    [np.abs(0.5 * s["m"] * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)).sum(),
                     np.abs(s["m"] * s["u"]).sum()] + [np.abs(s["m"]).sum() * 10.0] * 3)


def test_noalloc_diagnostics_matches_context_version():
    from paper_2005_02656_gb300 import SphSim
    L, lib = _lib()
    s = sph_inputs.jittered_box(30, seed_index=77, vel_sigma=0.3)
    sim = SphSim(s)
    ref = sim.diagnostics()                       # existing entry point (context scratch)
    scale = _scale(s)
    for call in range(2):
        out = np.full(8, np.nan)
        rc = lib.sph_diagnostics_noalloc(C.byref(sim._st), out.ctypes.data_as(C.c_void_p),
                                         _stream())
        assert rc == 0, (call, rc)
        np.testing.assert_allclose(out, ref, rtol=0, atol=1e-13 * scale.max())
        assert np.all(np.abs(out - ref) <= 1e-13 * scale), (call, out, ref)
    # a state larger than the static scratch is rejected
    big = L.SphState()
    big.n = N_MAX + 1
    for f in ("x", "y", "z", "vx", "vy", "vz", "m", "u"):
        setattr(big, f, sim.t["x"].data_ptr())
    out = np.zeros(8)
    assert lib.sph_diagnostics_noalloc(C.byref(big), out.ctypes.data_as(C.c_void_p),
                                       _stream()) == L.SPH_ERR_INVALID_ARG
    sim.close()


def test_noalloc_at_the_size_limit_then_a_small_state():
    """n = 16,777,216 uses every block slot of the static array; the small
    call after it shows the last block left the shared counter at zero."""
    import torch
    from paper_2005_02656_gb300 import SphSim
    L, lib = _lib()
    g = torch.Generator(device="cuda").manual_seed(12345)
    f = {k: torch.rand(N_MAX, dtype=torch.float64, device="cuda", generator=g) - 0.5
         for k in ("x", "y", "z", "vx", "vy", "vz")}
    f["m"] = torch.rand(N_MAX, dtype=torch.float64, device="cuda", generator=g) + 0.5
    f["u"] = torch.rand(N_MAX, dtype=torch.float64, device="cuda", generator=g) + 1.0
    st = L.SphState()
    st.n = N_MAX
    for k, t in f.items():
        setattr(st, k, t.data_ptr())
    out = np.full(8, np.nan)
    assert lib.sph_diagnostics_noalloc(C.byref(st), out.ctypes.data_as(C.c_void_p),
                                       _stream()) == 0
    m, x, y, z, vx, vy, vz, u = (f[k] for k in ("m", "x", "y", "z", "vx", "vy", "vz", "u"))
    terms = [m * vx, m * vy, m * vz, 0.5 * m * (vx * vx + vy * vy + vz * vz), m * u,
             m * (y * vz - z * vy), m * (z * vx - x * vz), m * (x * vy - y * vx)]
    ref = np.array([float(t.sum()) for t in terms])
    scale = np.array([float(t.abs().sum()) for t in terms])
    assert np.all(np.abs(out - ref) <= 1e-12 * scale), (out, ref)
    del f, terms, m, x, y, z, vx, vy, vz, u
    torch.cuda.empty_cache()
    s = sph_inputs.jittered_box(20, seed_index=78, vel_sigma=0.3)
    sim = SphSim(s)
    ref = sim.diagnostics()
    out = np.full(8, np.nan)
    assert lib.sph_diagnostics_noalloc(C.byref(sim._st), out.ctypes.data_as(C.c_void_p),
                                       _stream()) == 0
    assert np.all(np.abs(out - ref) <= 1e-13 * _scale(s)), (out, ref)
    sim.close()


def test_capturing_stream_is_refused_and_the_capture_survives():
    """The entry point synchronises its stream, which a capture forbids: it
    must return SPH_ERR_INVALID_ARG on a capturing stream and leave the
    caller's capture valid (it completes and replays correctly)."""
    import torch
    from paper_2005_02656_gb300 import SphSim
    L, lib = _lib()
    s = sph_inputs.jittered_box(12, seed_index=79, vel_sigma=0.3)
    sim = SphSim(s)
    out = np.zeros(8)
    assert lib.sph_diagnostics_noalloc(C.byref(sim._st), out.ctypes.data_as(C.c_void_p),
                                       _stream()) == 0
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    out2 = np.zeros(8)
    with torch.cuda.graph(graph):
        rc = lib.sph_diagnostics_noalloc(C.byref(sim._st), out2.ctypes.data_as(C.c_void_p),
                                         _stream())
        y = x * 3.0
    assert rc == L.SPH_ERR_INVALID_ARG
    x.copy_(torch.arange(1000, dtype=torch.float64, device="cuda") + 1.0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(y, (torch.arange(1000, dtype=torch.float64, device="cuda") + 1.0) * 3.0)
    again = np.zeros(8)
    assert lib.sph_diagnostics_noalloc(C.byref(sim._st), again.ctypes.data_as(C.c_void_p),
                                       _stream()) == 0
    np.testing.assert_array_equal(again, out)
    sim.close()
