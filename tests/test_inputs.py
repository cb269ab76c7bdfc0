"""The synthetic workloads (sph_inputs): seeded, of the sizes the benchmark
and the tests quote, and with the structure their recipes state."""
import math

import numpy as np
import pytest

import sph_inputs


def _same(a, b):
    for k in ("x", "y", "z", "vx", "vy", "vz", "h", "m", "u", "id"):
        np.testing.assert_array_equal(a[k], b[k])


def test_generators_are_seeded():
    _same(sph_inputs.jittered_box(12, seed_index=9), sph_inputs.jittered_box(12, seed_index=9))
    a = sph_inputs.jittered_box(12, seed_index=9)
    b = sph_inputs.jittered_box(12, seed_index=10)
    assert not np.array_equal(a["x"], b["x"])


def test_jittered_box_recipe():
    s = sph_inputs.jittered_box(20)
    n = 20 ** 3
    assert s["x"].shape == (n,) and s["periodic"] == (1, 1, 1)
    np.testing.assert_allclose(s["m"], 1.0 / n)
    np.testing.assert_array_equal(s["u"], 1.0)
    lattice = (np.sort(s["id"]) == np.arange(n)).all()
    assert lattice
    # jitter within 0.1 spacing of the lattice sites (i + 1/2) / 20
    order = np.argsort(s["id"])
    x = s["x"][order]
    site = (np.floor(x * 20) + 0.5) / 20
    assert np.abs(x - site).max() <= 0.1 / 20 + 1e-15
    assert s["h"][0] == pytest.approx(sph_inputs.h_for_neighbors(1.0 / 20))
    assert 0.005 < s["vx"].std() < 0.015
    np.testing.assert_array_equal(s["vx"], s["vxh"])
    np.testing.assert_array_equal(s["du_prev"], 0.0)


def test_square_patch_recipe():
    s = sph_inputs.square_patch(20)
    assert s["x"].shape == (8000,) and s["periodic"] == (0, 0, 1)
    np.testing.assert_allclose(s["vx"], 5.0 * s["y"])
    np.testing.assert_allclose(s["vy"], -5.0 * s["x"])
    np.testing.assert_allclose(s["m"].sum(), 1.0)          # density 1 in the unit cube


def test_kelvin_helmholtz_size_and_layers():
    s = sph_inputs.kelvin_helmholtz(224)
    n = s["x"].shape[0]
    assert n == 8_416_298
    inner = (s["y"] >= 0.25) & (s["y"] < 0.75)
    # equal-mass particles within 0.24%, twice as many per volume inside
    m_in, m_out = s["m"][inner].mean(), s["m"][~inner].mean()
    assert abs(m_in / m_out - 1) < 0.0025
    assert inner.sum() / (~inner).sum() == pytest.approx(2.0, rel=0.01)
    np.testing.assert_allclose(s["vx"][inner], 0.5)
    np.testing.assert_allclose(s["vx"][~inner], -0.5)
    np.testing.assert_allclose(s["vy"], 0.01 * np.sin(4 * math.pi * s["x"]))
    # uniform pressure 2.5 with gamma = 5/3: u = 3.75 / rho
    np.testing.assert_allclose(s["u"][inner], 3.75 / 2)
    np.testing.assert_allclose(s["u"][~inner], 3.75)


def test_ensemble_sizes():
    sides, alphas = sph_inputs.ensemble_sides()
    assert sides.shape == (256,) and sides.min() >= 8 and sides.max() <= 48
    assert int((sides ** 3).sum()) == 5_030_778
    assert 0.5 <= alphas.min() and alphas.max() <= 1.5


def test_uniform_sphere_size():
    s = sph_inputs.uniform_sphere(124, seed_index=83)   # the self-gravity benchmark's sphere
    assert s["x"].shape[0] == 998_317
    r = np.sqrt(s["x"] ** 2 + s["y"] ** 2 + s["z"] ** 2)
    assert r.max() < 1.0 + 0.1 * 2 / 124
    np.testing.assert_allclose(s["m"].sum(), 1.0)
    assert s["periodic"] == (0, 0, 0)
