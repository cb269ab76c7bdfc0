"""Parity at full workload sizes, in the configuration bench.py times, on
sampled particles the oracle computes one by one (oracle.sampled_outputs:
density on the 2-ring of the sample, IAD on its 1-ring, momentum on the
sample).

* Rotating square patch, 100^3 = 10^6 particles (x, y open, z periodic),
  FP64, 10 steps: at steps 0, 4 and 9 the GPU's pre-step state is handed to
  the oracle and the step's outputs are compared on a sample (the two
  trajectories separate at rounding level, so each step is checked on
  identical inputs).
* Kelvin-Helmholtz box, 8,416,298 particles: one FP64 and one FP32-mixed step;
  the sampled particles' neighbour lists (exact in both precisions), density,
  IAD matrix C, accelerations and du.
"""
import numpy as np
import pytest

import oracle
import sph_inputs
from helpers import sym

pytestmark = pytest.mark.gpu

# FP32-mixed C: max_ij |C - C_ref| / max_ij |C_ref| per particle; tau is a sum
# of ~100 FP32 terms on 1/h-scaled separations (relative ~1e-6) and the
# cofactor inverse multiplies by the condition number of tau (<~ 10 on these
# lattices)
FP32_IAD_TOL = 1e-4


def _sample_errors(got, ref, sample_ids):
    e = {}
    e["rho"] = np.max(np.abs(got["rho"][sample_ids] - ref["rho"]) / ref["rho"])
    a_g = np.stack([got[k][sample_ids] for k in ("ax", "ay", "az")], 1)
    a_r = np.stack([ref[k] for k in ("ax", "ay", "az")], 1)
    e["a"] = np.max(np.abs(a_g - a_r).max(1) / ref["sa"])
    e["du"] = np.max(np.abs(got["du"][sample_ids] - ref["du"]) / np.maximum(ref["sdu"], 1e-300))
    C = ref["iad"]
    e["iad"] = np.max(np.abs(got["iad"][sample_ids] - C).max(1) / np.abs(C).max(1))
    return e


def _pre_step_by_id(sim):
    s = sim.to_numpy(by_id=True)
    return {k: s[k] for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m",
                              "u", "du_prev", "id")}


def _check_step(sim, state_before, box, params, sample, tol, max_nb):
    """Compare the outputs of the step just taken with the oracle's on
    `state_before` (ordered by id) for the sampled ids."""
    rc, ref = oracle.sampled_outputs(box, state_before, params, sample)
    assert rc == 0
    got = sim.to_numpy(by_id=True)
    e = _sample_errors(got, ref, sample)
    for k, t in tol.items():
        assert e[k] <= t, (k, e)
    return e


def _lists_for_sample(sim, sample):
    counts, ids = sim.get_neighbors()
    cur_id = sim.t["id"].cpu().numpy()
    counts, ids = counts.cpu().numpy(), ids.cpu().numpy()
    pos = np.empty_like(cur_id)
    pos[cur_id] = np.arange(cur_id.shape[0])
    return counts[pos[sample]], ids[pos[sample]]


def test_square_patch_1m_ten_steps_fp64():
    from paper_2005_02656_gb300 import SphSim
    s = sph_inputs.square_patch(100)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    params = oracle.Params()
    sim = SphSim(s)
    rng = np.random.default_rng(5)
    tol = {"rho": 1e-12, "a": 1e-12, "du": 1e-12}
    for step in range(10):
        check = step in (0, 4, 9)
        if check:
            before = _pre_step_by_id(sim)
            # neighbour lists of the pre-step state, sampled, must match exactly
            sim.find_neighbors()
            sample = rng.choice(before["x"].shape[0], 300, replace=False)
            counts, ids = _lists_for_sample(sim, sample)
            rc, nn_ref, nbr_ref = oracle.find_neighbors(box, before["x"], before["y"], before["z"],
                                                       before["h"], targets=sample,
                                                       max_nb=params.max_nb)
            assert rc == 0
            np.testing.assert_array_equal(counts, nn_ref)
            for i in range(sample.shape[0]):
                np.testing.assert_array_equal(ids[i, :counts[i]], nbr_ref[i, :counts[i]])
        sim.step()
        if check:
            before_sorted = {k: v for k, v in before.items()}
            before_sorted.update(lo=s["lo"], hi=s["hi"], periodic=s["periodic"])
            _check_step(sim, before_sorted, box, params, sample, tol, params.max_nb)
    assert sim.error_word() == 0
    # the patch stays bounded and spins (angular momentum about z keeps its sign)
    d = sim.diagnostics()
    assert d[7] < 0 and np.isfinite(d).all()
    sim.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_kelvin_helmholtz_8m_sampled(precision):
    from paper_2005_02656_gb300 import SphSim
    s = sph_inputs.kelvin_helmholtz(224)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    params = oracle.Params()
    sim = SphSim(s, precision=precision)
    before = _pre_step_by_id(sim)
    before.update(lo=s["lo"], hi=s["hi"], periodic=s["periodic"])
    rng = np.random.default_rng(6)
    sample = rng.choice(before["x"].shape[0], 200, replace=False)
    # the search of the step's pre-step state: sampled lists bit-exact
    sim.find_neighbors()
    counts, ids = _lists_for_sample(sim, sample)
    rc, nn_ref, nbr_ref = oracle.find_neighbors(box, before["x"], before["y"], before["z"],
                                               before["h"], targets=sample, max_nb=params.max_nb)
    assert rc == 0
    np.testing.assert_array_equal(counts, nn_ref)
    for i in range(sample.shape[0]):
        np.testing.assert_array_equal(ids[i, :counts[i]], nbr_ref[i, :counts[i]])
    sim.step()
    assert sim.error_word() == 0
    tol = ({"rho": 1e-12, "iad": 1e-12, "a": 1e-12, "du": 1e-12} if precision == "fp64"
           else {"rho": 1e-5, "iad": FP32_IAD_TOL, "a": 1e-4, "du": 1e-4})
    _check_step(sim, before, box, params, sample, tol, params.max_nb)
    sim.close()
