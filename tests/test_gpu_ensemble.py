"""The batched ensemble (one persistent cooperative launch for all boxes):
each box matches a separate single-box run of the same device code, the CUDA
graph replay matches eager launches, the bounded grid barrier reports a
timeout instead of hanging and leaves the context usable, and the autotuner
returns a valid configuration."""
import numpy as np
import pytest

import oracle
import sph_inputs

pytestmark = pytest.mark.gpu

SIDES = (7, 8, 9, 12, 16, 20, 24)


def _boxes():
    return [(sph_inputs.jittered_box(s, seed_index=300 + i, vel_sigma=0.2), 0.5 + 0.15 * i)
            for i, s in enumerate(SIDES)]


def test_each_box_matches_its_single_box_run():
    from paper_2005_02656_gb300 import Ensemble, SphSim
    boxes = _boxes()
    ens = Ensemble(boxes)
    ens.step(3)
    assert ens.error_word() == 0
    for b, (s, alpha) in enumerate(boxes):
        sim = SphSim(s, precision="fp32_mixed", alpha=alpha, pair_mode="lists")
        sim.step(3)
        ref = sim.to_numpy()
        got = ens.box_numpy(b)
        for k in ("x", "y", "z", "vx", "u", "h", "rho", "ax", "du"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"box {b} field {k}")
        np.testing.assert_allclose(ens.dt.cpu().numpy()[b], sim.dt.cpu().numpy()[0], rtol=0)
        sim.close()
    ens.close()


def test_ensemble_box_against_oracle():
    """One box of the ensemble, first step, against the FP64 oracle (FP32-mixed tolerances)."""
    from paper_2005_02656_gb300 import Ensemble
    boxes = _boxes()
    ens = Ensemble(boxes)
    ens.step(1)
    b = 5
    s, alpha = boxes[b]
    ref_s = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    order = np.argsort(ref_s["id"])
    ref_s = {k: (v[order] if isinstance(v, np.ndarray) else v) for k, v in ref_s.items()}
    rc, out = oracle.outputs(oracle.Box(s["lo"], s["hi"], s["periodic"]), ref_s,
                             oracle.Params(alpha=alpha))
    assert rc == 0
    got = ens.box_numpy(b)
    assert np.max(np.abs(got["rho"] - out["rho"]) / out["rho"]) < 1e-5
    a_g = np.stack([got["ax"], got["ay"], got["az"]], 1)
    a_r = np.stack([out["ax"], out["ay"], out["az"]], 1)
    assert np.max(np.abs(a_g - a_r).max(1) / out["sa"]) < 1e-4
    assert np.max(np.abs(got["du"] - out["du"]) / out["sdu"]) < 1e-4
    ens.close()


def test_graph_replay_matches_eager():
    from paper_2005_02656_gb300 import Ensemble
    boxes = _boxes()
    eager = Ensemble(boxes)
    eager.step(2)
    eager.step(2)
    e = eager.box_numpy(6)
    eager.close()
    g = Ensemble(boxes)
    g.capture(2)
    g.replay()
    g.replay()
    g.synchronize()
    assert g.error_word() == 0
    r = g.box_numpy(6)
    for k in ("x", "vx", "u", "h", "rho"):
        np.testing.assert_array_equal(r[k], e[k])
    g.close()


def test_barrier_timeout_is_reported_and_context_recovers():
    """A CTA that never arrives (test hook) makes the others' bounded wait
    expire: SPH_FLAG_TIMEOUT is raised, the kernel returns, and after reading
    the error word the ensemble steps normally."""
    from paper_2005_02656_gb300 import Ensemble, _lib
    ens = Ensemble(_boxes())
    ens.set_config(test_skip_block=0)
    ens.step(1)
    assert ens.error_word() & _lib.FLAG_TIMEOUT
    ens.set_config(test_skip_block=-1)
    ens.step(1)
    assert ens.error_word() == 0
    ens.close()


@pytest.mark.parametrize("find_window,tpp,tpm", [(128, 1, 1), (256, 2, 2), (512, 4, 4), (256, 1, 4)])
def test_tile_shape_and_threads_per_particle_against_oracle(find_window, tpp, tpm):
    """Every tile shape and thread count gives the same neighbour sets and
    sums within the FP32-mixed tolerances (the split changes only the
    summation order)."""
    from paper_2005_02656_gb300 import Ensemble
    boxes = _boxes()
    ens = Ensemble(boxes)
    ens.set_config(find_window=find_window, threads_per_particle=tpp, momentum_threads=tpm)
    ens.step(1)
    assert ens.error_word() == 0
    for b in (0, 5):
        s, alpha = boxes[b]
        order = np.argsort(s["id"])
        ref_s = {k: (v[order] if isinstance(v, np.ndarray) else v) for k, v in s.items()}
        rc, out = oracle.outputs(oracle.Box(s["lo"], s["hi"], s["periodic"]), ref_s,
                                 oracle.Params(alpha=alpha))
        assert rc == 0
        got = ens.box_numpy(b)
        assert np.max(np.abs(got["rho"] - out["rho"]) / out["rho"]) < 1e-5
        a_g = np.stack([got["ax"], got["ay"], got["az"]], 1)
        a_r = np.stack([out["ax"], out["ay"], out["az"]], 1)
        assert np.max(np.abs(a_g - a_r).max(1) / out["sa"]) < 1e-4
        assert np.max(np.abs(got["du"] - out["du"]) / out["sdu"]) < 1e-4
    ens.close()


def test_bad_config_is_rejected():
    from paper_2005_02656_gb300 import Ensemble, _lib
    ens = Ensemble(_boxes()[:2])
    with pytest.raises(_lib.SphError):
        ens.set_config(find_window=200)
    with pytest.raises(_lib.SphError):
        ens.set_config(find_window=512, threads_per_particle=3)
    with pytest.raises(_lib.SphError):
        ens.set_config(threads_per_particle=1, momentum_threads=3)
    ens.close()
    s = sph_inputs.jittered_box(8, seed_index=310)
    empty = {k: (v[:0].copy() if isinstance(v, np.ndarray) else v) for k, v in s.items()}
    with pytest.raises(_lib.SphError) as e:
        Ensemble([(s, 1.0), (empty, 1.0)])
    assert e.value.code == _lib.SPH_ERR_INVALID_ARG


def test_autotune_picks_a_configuration():
    from paper_2005_02656_gb300 import Ensemble
    ens = Ensemble(_boxes())
    before = ens.box_numpy(3)
    res = ens.autotune(steps=1, cell_factors=(1.0, 1.3), find_windows=(128, 512),
                       threads_per_particle=(1, 2), momentum_threads=(4, 2))
    assert res["cell_factor"] in (1.0, 1.3) and res["seconds_per_step"] > 0
    assert res["find_window"] in (128, 512) and res["threads_per_particle"] in (1, 2)
    assert res["momentum_threads"] in (4, 2)
    assert len(res["tried"]) == 6
    after = ens.box_numpy(3)
    np.testing.assert_array_equal(before["x"], after["x"])   # tuning leaves the state alone
    ens.step(1)
    assert ens.error_word() == 0
    ens.close()


def test_gradh_boxes_match_their_single_box_runs():
    """With the grad-h terms on (Omega in X = P / (Omega rho^2)), each box of
    the ensemble still equals its own single-box FP32-mixed run bit for bit."""
    from paper_2005_02656_gb300 import Ensemble, Params, SphSim
    boxes = _boxes()[:4]
    ens = Ensemble(boxes, Params(precision="fp32_mixed", gradh=1))
    ens.step(2)
    assert ens.error_word() == 0
    for b, (s, alpha) in enumerate(boxes):
        sim = SphSim(s, precision="fp32_mixed", alpha=alpha, gradh=1, pair_mode="lists")
        sim.step(2)
        ref = sim.to_numpy()
        got = ens.box_numpy(b)
        for k in ("x", "vx", "u", "h", "rho", "ax", "du"):
            np.testing.assert_array_equal(got[k], ref[k], err_msg=f"box {b} field {k}")
        sim.close()
    ens.close()
