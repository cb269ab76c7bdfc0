"""Self-gravity on the GPU (sph_gravity): the multipole tree on the
neighbour grid's cells against the oracle's tree (same reading, same
acceptance decisions, so the sums agree to FP64 rounding and the interaction
counts exactly) and against the exact direct sum (the approximation error of
the quadrupole expansion at theta = 0.5).  The FP32-mixed walk takes the same
decisions (equal interaction counts) and agrees within the FP32 acceleration
tolerance, 1e-4 of max|g|."""
import numpy as np
import pytest

import oracle
import sph_inputs

pytestmark = pytest.mark.gpu

EPS = 1e-3
TOL32 = 1e-4     # FP32-mixed acceleration tolerance, relative to max |g|


def _gpu(s, theta, G=1.0, eps=EPS, precision="fp64"):
    from paper_2005_02656_gb300 import Params, SphSim
    sim = SphSim(s, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                           precision=precision))
    g, counts = sim.gravity(G, eps, theta)
    g = g.cpu().numpy()
    ids = sim.t["id"].cpu().numpy()
    assert sim.error_word() == 0
    sim.close()
    out = np.empty_like(g)
    out[ids] = g                  # back to id order
    return out, counts


def _by_id(s):
    order = np.argsort(s["id"])
    return {k: (v[order] if isinstance(v, np.ndarray) else v) for k, v in s.items()}


@pytest.mark.parametrize("theta,eps", [(0.0, EPS), (0.5, EPS), (0.8, EPS), (0.5, 0.0)])
def test_tree_matches_oracle_tree(theta, eps):
    s = sph_inputs.uniform_sphere(22, seed_index=81)
    g, counts = _gpu(s, theta, eps=eps)
    # the oracle sees the arrays in the order the GPU received them
    rc, ref, st = oracle.gravity_tree(s, eps=eps, theta=theta)
    assert rc == 0
    ref_by_id = np.empty_like(ref)
    ref_by_id[s["id"]] = ref
    scale = np.abs(ref_by_id).max()
    assert np.abs(g - ref_by_id).max() <= 1e-12 * scale
    np.testing.assert_array_equal(counts, st)


@pytest.mark.parametrize("theta,eps", [(0.0, EPS), (0.5, EPS), (0.8, EPS), (0.5, 0.0)])
def test_fp32_matches_oracle_tree(theta, eps):
    s = sph_inputs.uniform_sphere(22, seed_index=81)
    g, counts = _gpu(s, theta, eps=eps, precision="fp32_mixed")
    rc, ref, st = oracle.gravity_tree(s, eps=eps, theta=theta)
    assert rc == 0
    ref_by_id = np.empty_like(ref)
    ref_by_id[s["id"]] = ref
    scale = np.abs(ref_by_id).max()
    err = np.abs(g - ref_by_id).max() / scale
    assert err <= TOL32, err
    assert err > 0.0           # FP32 arithmetic did run
    np.testing.assert_array_equal(counts, st)


def test_fp32_decisions_on_an_exact_lattice():
    """Unjittered lattice points lie on cell faces and at equal distances, so
    many FP32 decisions fall inside the margin and are taken in FP64: the
    counts still equal the FP64 walk's."""
    s = sph_inputs.uniform_sphere(24, seed_index=85, jitter=0.0)
    g64, c64 = _gpu(s, 0.5)
    g32, c32 = _gpu(s, 0.5, precision="fp32_mixed")
    np.testing.assert_array_equal(c32, c64)
    assert np.abs(g32 - g64).max() <= TOL32 * np.abs(g64).max()


def test_tree_error_against_direct_sum():
    s = sph_inputs.uniform_sphere(22, seed_index=82)
    g, _ = _gpu(s, 0.5)
    d = oracle.gravity_direct(_by_id(s), eps=EPS)
    e = np.linalg.norm(g - d, axis=1) / np.linalg.norm(d, axis=1)
    assert np.sqrt((e ** 2).mean()) < 1e-3 and e.max() < 1e-2


def test_full_size_sampled():
    """About 10^6 particles: sampled targets against the oracle's tree (exact
    agreement) and the direct sum (approximation error)."""
    s = sph_inputs.uniform_sphere(124, seed_index=83)
    n = s["x"].shape[0]
    assert n > 990_000
    g, counts = _gpu(s, 0.5)
    rng = np.random.default_rng(4)
    sample_ids = rng.choice(n, 300, replace=False)
    pos = np.empty(n, dtype=np.int64)
    pos[s["id"]] = np.arange(n)             # array position of each id
    rc, ref, st = oracle.gravity_tree(s, eps=EPS, theta=0.5, targets=pos[sample_ids])
    assert rc == 0
    assert np.abs(g[sample_ids] - ref).max() <= 1e-12 * np.abs(ref).max()
    d = oracle.gravity_direct(s, eps=EPS, targets=pos[sample_ids])
    e = np.linalg.norm(g[sample_ids] - d, axis=1) / np.linalg.norm(d, axis=1)
    assert np.sqrt((e ** 2).mean()) < 1e-3
    assert counts[0] > 0 and counts[1] > 0


def test_fp32_full_size_sampled():
    s = sph_inputs.uniform_sphere(124, seed_index=83)
    n = s["x"].shape[0]
    g, counts = _gpu(s, 0.5, precision="fp32_mixed")
    rng = np.random.default_rng(5)
    sample_ids = rng.choice(n, 300, replace=False)
    pos = np.empty(n, dtype=np.int64)
    pos[s["id"]] = np.arange(n)
    rc, ref, _ = oracle.gravity_tree(s, eps=EPS, theta=0.5, targets=pos[sample_ids])
    assert rc == 0
    assert np.abs(g[sample_ids] - ref).max() <= TOL32 * np.abs(ref).max()
    g64, c64 = _gpu(s, 0.5)
    np.testing.assert_array_equal(counts, c64)
    assert np.abs(g - g64).max() <= TOL32 * np.abs(g64).max()


def test_periodic_box_is_rejected():
    from paper_2005_02656_gb300 import SphSim, _lib
    s = sph_inputs.jittered_box(8, seed_index=84)
    sim = SphSim(s)
    with pytest.raises(_lib.SphError) as e:
        sim.gravity()
    assert e.value.code == _lib.SPH_ERR_INVALID_ARG
    sim.close()


def _few(xyz, m, h=0.1):
    n = len(m)
    s = {k: np.zeros(n) for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh",
                                  "du_prev")}
    s["x"], s["y"], s["z"] = (np.array(c, dtype=np.float64) for c in zip(*xyz)) if n else \
        (np.zeros(0), np.zeros(0), np.zeros(0))
    s["m"] = np.asarray(m, dtype=np.float64)
    s["h"] = np.full(n, h)
    s["u"] = np.ones(n)
    s["id"] = np.arange(n, dtype=np.int64)
    s["lo"], s["hi"], s["periodic"] = (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (0, 0, 0)
    return s


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_two_bodies_closed_form(precision):
    """Two bodies 0.5 apart along a diagonal: the softened Newtonian pull,
    equal and opposite momentum (the leaves are opened, so the sum is direct)."""
    s = _few([(0.1, 0.2, 0.3), (0.4, 0.6, 0.3)], [2.0, 0.5])
    G, eps = 1.5, 0.1
    g, counts = _gpu(s, 0.5, G=G, eps=eps, precision=precision)
    d = np.array([0.3, 0.4, 0.0])
    f = G / (0.25 + eps * eps) ** 1.5
    tol = 1e-14 if precision == "fp64" else 1e-6
    np.testing.assert_allclose(g[0], f * 0.5 * d, rtol=tol, atol=tol * f)
    np.testing.assert_allclose(g[1], -f * 2.0 * d, rtol=tol, atol=tol * f)
    assert counts[1] == 2


@pytest.mark.parametrize("precision", ["fp64", "fp32_mixed"])
def test_single_particle_and_empty(precision):
    g, counts = _gpu(_few([(0.1, 0.2, 0.3)], [1.0]), 0.5, precision=precision)
    np.testing.assert_array_equal(g, np.zeros((1, 3)))
    np.testing.assert_array_equal(counts, [0, 0])
    from paper_2005_02656_gb300 import Params, SphSim
    s = _few([], [])
    sim = SphSim(s, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                           precision=precision), n_max=4)
    g, counts = sim.gravity(1.0, EPS, 0.5)
    assert g.shape == (0, 3)
    np.testing.assert_array_equal(counts, [0, 0])
    assert sim.error_word() == 0
    sim.close()
