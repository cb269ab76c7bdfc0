"""GPU behaviour beyond parity: error flags raised from host-made faults (no
GPU fault is provoked), argument checks, call order, determinism,
conservation to rounding, the host-buffer step and the diagnostics."""
import ctypes as C
import math

import numpy as np
import pytest

import oracle
import sph_inputs

pytestmark = pytest.mark.gpu


def _sim(s, **kw):
    from paper_2005_02656_gb300 import SphSim
    return SphSim(s, **kw)


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_neighbor_overflow_flag_and_true_counts(precision):
    from paper_2005_02656_gb300 import _lib
    s = sph_inputs.jittered_box(16, seed_index=40)
    sim = _sim(s, max_nb=32, ng_target=0, precision=precision)
    sim.find_neighbors()
    counts, _ = sim.get_neighbors()
    assert sim.error_word() & _lib.FLAG_NB_OVERFLOW
    assert counts.max().item() > 32          # true counts are kept
    sim.close()


def test_bad_box_flag():
    from paper_2005_02656_gb300 import _lib
    s = sph_inputs.jittered_box(8, seed_index=41)
    s["h"][:] = 0.3                          # 2h >= L/2 on periodic axes
    sim = _sim(s, ng_target=0)
    sim.find_neighbors()
    assert sim.error_word() & _lib.FLAG_BAD_BOX
    sim.close()


def test_nonfinite_input_is_flagged():
    from paper_2005_02656_gb300 import _lib
    s = sph_inputs.jittered_box(12, seed_index=42)
    s["u"][5] = np.nan                       # NaN planted on the host
    sim = _sim(s, ng_target=0)
    sim.step()
    assert sim.error_word() & _lib.FLAG_NONFINITE
    sim.close()


def test_argument_and_order_errors():
    from paper_2005_02656_gb300 import _lib
    s = sph_inputs.jittered_box(8, seed_index=43)
    sim = _sim(s)
    with pytest.raises(_lib.SphError) as e:
        sim.density()                        # no lists yet
    assert e.value.code == _lib.SPH_ERR_ORDER
    sim.find_neighbors()
    with pytest.raises(_lib.SphError) as e:
        sim.momentum_energy()                # IAD missing
    assert e.value.code == _lib.SPH_ERR_ORDER
    big = _lib.SphState()
    big.n = sim.n_max + 1
    rc = sim.lib.sph_step(sim.ctx, C.byref(big), C.c_void_p(sim.dt.data_ptr()), None)
    assert rc == _lib.SPH_ERR_INVALID_ARG
    assert b"n_max" in sim.lib.sph_last_error(sim.ctx)
    sim.close()
    p = _lib.SphParams()
    sim.lib.sph_default_params(C.byref(p))
    p.max_nb = 30                            # not a multiple of 4
    ctx = C.c_void_p()
    assert sim.lib.sph_init(C.byref(p), 100, C.byref(ctx)) == _lib.SPH_ERR_INVALID_ARG


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_two_runs_bit_identical(precision):
    s = sph_inputs.jittered_box(20, seed_index=44, vel_sigma=0.2)
    outs = []
    for _ in range(2):
        sim = _sim(s, precision=precision)
        sim.step(3)
        outs.append(sim.to_numpy())
        sim.close()
    for k in ("x", "vx", "u", "h", "rho", "ax", "du"):
        np.testing.assert_array_equal(outs[0][k], outs[1][k])


def test_conservation_to_rounding_common_h():
    """With one smoothing length the lists are symmetric, so the step's pair
    sums conserve momentum and energy exactly up to rounding (Eqs. 2-4)."""
    s = sph_inputs.jittered_box(20, seed_index=45, vel_sigma=0.3)
    sim = _sim(s, ng_target=0)
    sim.find_neighbors()
    sim.density()
    sim.iad()
    sim.momentum_energy()
    g = sim.to_numpy()
    m = g["m"]
    a = np.stack([g["ax"], g["ay"], g["az"]], 1)
    v = np.stack([g["vx"], g["vy"], g["vz"]], 1)
    scale = (m[:, None] * np.abs(a)).sum() + 1e-300
    # reference scale from the oracle (sum of |pair terms|)
    rc, ref = oracle.outputs(oracle.Box(s["lo"], s["hi"], s["periodic"]),
                             {k: g[k] for k in ("x", "y", "z", "vx", "vy", "vz", "h", "m", "u")},
                             oracle.Params(ng_target=0))
    S = (m * ref["sa"]).sum()
    assert np.abs((m[:, None] * a).sum(0)).max() < 1e-13 * S
    power = (m * ((v * a).sum(1) + g["du"])).sum()
    assert abs(power) < 1e-13 * (m * (np.linalg.norm(v, axis=1) * ref["sa"] + ref["sdu"])).sum()
    assert scale > 0
    sim.close()


@pytest.mark.parametrize("precision,side,pinned", [("fp32_mixed", 16, True), ("fp32_mixed", 27, True),
                                                   ("fp64", 19, True), ("fp32_mixed", 17, False)])
def test_host_step_equals_device_step(precision, side, pinned):
    """sph_step_host on pinned host arrays gives the device step's results,
    step after step: its copies run on two streams (positions first, m, u, id
    and then the velocities and integrator history while the sort and search
    run; m, id and du_prev copied out early; with pinned arrays the update
    kernel writes the rest straight into them, with pageable ones they are
    copied), so every field is checked."""
    from paper_2005_02656_gb300 import HostStepper, Params
    s = sph_inputs.jittered_box(side, seed_index=46, vel_sigma=0.1)
    steps = 3
    dev = _sim(s, precision=precision)
    dev.step(steps)
    d = dev.to_numpy()
    dev.close()
    hs = HostStepper(s, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                               precision=precision), outputs=True, pinned=pinned)
    for _ in range(steps):
        hs.step()
    h = {k: v.numpy() for k, v in hs.h.items()}
    order = np.argsort(h["id"])
    np.testing.assert_array_equal(h["id"][order], np.arange(side ** 3))
    for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "u", "du_prev", "h", "m",
              "rho", "ax", "du"):
        np.testing.assert_array_equal(h[k][order], d[k], err_msg=k)
    hs.close()


@pytest.mark.parametrize("angular", [1, 0])
def test_diagnostics_match_numpy_and_last_step(angular):
    s = sph_inputs.jittered_box(14, seed_index=47, vel_sigma=0.4)
    sim = _sim(s, angular_sums=angular)
    d0 = sim.diagnostics()
    m = s["m"]
    assert d0[0] == pytest.approx(math.fsum(m * s["vx"]), abs=1e-15)
    assert d0[3] == pytest.approx(math.fsum(0.5 * m * (s["vx"] ** 2 + s["vy"] ** 2 + s["vz"] ** 2)),
                                  rel=1e-13)
    assert d0[4] == pytest.approx(math.fsum(m * s["u"]), rel=1e-13)
    sim.step()
    last = sim.last_diagnostics()
    now = sim.diagnostics()
    if angular:
        np.testing.assert_allclose(last[:8], now, rtol=1e-13, atol=1e-16)
    else:  # momentum and energy are always summed; angular momentum only on request
        np.testing.assert_allclose(last[:5], now[:5], rtol=1e-13, atol=1e-16)
        assert np.isnan(last[5:8]).all()
    g = sim.to_numpy()
    assert last[8] == pytest.approx(float(sim.dt.cpu()[0]))
    assert last[9] >= 1 and last[10] >= last[9]
    sim.close()


def test_profile_and_counters():
    s = sph_inputs.jittered_box(16, seed_index=48)
    sim = _sim(s, precision="fp32_mixed")
    sim.profile(True)
    sim.step(2)
    times, steps = sim.stage_times()
    assert steps == 2 and all(v >= 0 for v in times.values()) and times["find"] > 0
    st = sim.stats()
    assert st["pairs"] > 0 and st["candidates"] > st["pairs"] and st["particle_updates"] == 2 * sim.n
    assert sim.launch_count() > 0
    sim.close()


def test_precision_switch_to_fp64_allocates_its_cache():
    """A context created FP32-mixed and switched to FP64 by set_params gets
    the FP64 path's per-entry kernel cache and then matches the oracle to the
    FP64 tolerance."""
    from helpers import field_errors, oracle_outputs
    s = sph_inputs.jittered_box(12, seed_index=49, vel_sigma=0.2)
    sim = _sim(s, precision="fp32_mixed", ng_target=0)
    sim.set_params(precision="fp64")
    sim.find_neighbors()
    sim.density()
    sim.iad()
    sim.momentum_energy()
    got = sim.to_numpy()
    assert sim.error_word() == 0
    sim.close()
    rc, _, ref = oracle_outputs(s, ng_target=0)
    assert rc == 0
    e = field_errors(got, ref)
    for k in ("rho", "iad", "a", "du"):
        assert e[k] <= 1e-12, (k, e)
