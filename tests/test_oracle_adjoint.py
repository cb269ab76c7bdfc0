"""Pins of the reference adjoint (oracle/adjoint.py) on the CPU.

The reference adjoint is reverse-mode AD of a PyTorch FP64 restatement of K
frozen steps.  It is pinned here by things other than itself:
  * its forward values equal the C oracle's frozen rollout (which reproduces
    the C oracle's own base run bit for bit);
  * its gradient equals central differences of the C oracle's frozen rollout
    (lists, h, dt and the viscosity switch of Eq. 5 held fixed);
  * forward-mode (dual-number) derivatives equal the reverse-mode ones;
  * closed forms from the symmetries of the method: a uniform translation of
    every position leaves the loss unchanged (periodic box, minimum image), so
    sum_a dL/dx_a = 0; a uniform velocity shift e moves every particle by
    e t and leaves every pair quantity unchanged, so
    sum_a dL/dv_a . e = sum_a m_a v_a(K) . e.
"""
import numpy as np
import pytest

import oracle
import sph_inputs
from oracle import adjoint as adj

K = 4


@pytest.fixture(scope="module")
def case():
    s = sph_inputs.jittered_box(10, seed_index=70, vel_sigma=0.05)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    prm = oracle.Params()
    tape = adj.record(box, s, prm, K)
    g = adj.reference_gradients(box, s, prm, tape)
    return s, box, prm, tape, g


def test_frozen_rollout_reproduces_base_run(case):
    s, box, prm, tape, _ = case
    base = oracle.copy_state(s)
    dt_prev = 0.0
    for _ in range(K):
        rc, dt, _ = oracle.step(box, base, prm, dt_prev)
        assert rc == oracle.OK
        dt_prev = dt
    _, fin, _ = adj.frozen_loss(box, s, prm, tape)
    for k in ("x", "y", "z", "vx", "vy", "vz", "u", "h"):
        np.testing.assert_array_equal(fin[k], base[k])


def test_torch_forward_equals_c_oracle(case):
    s, box, prm, tape, _ = case
    L, fin, rho = adj.frozen_loss(box, s, prm, tape)
    x0, v0, u0, al = adj._inputs(s, prm.alpha)
    x, v, u, r = adj.torch_rollout(box, s, prm, tape, x0, v0, al, u0=u0)
    np.testing.assert_allclose(x.numpy(), np.stack([fin["x"], fin["y"], fin["z"]], 1),
                               rtol=0, atol=1e-14)
    vr = np.stack([fin["vx"], fin["vy"], fin["vz"]], 1)
    assert np.abs(v.numpy() - vr).max() <= 1e-12 * np.abs(vr).max()
    np.testing.assert_allclose(u.numpy(), fin["u"], rtol=1e-13)
    np.testing.assert_allclose(r.numpy(), rho, rtol=1e-13)
    assert float(adj.torch_loss(r, v, adj.torch.as_tensor(s["m"]))) == pytest.approx(L, rel=1e-13)


def _fd(box, s, prm, tape, dx, dv, du, da, eps):
    """Central difference of the C oracle's frozen loss along (dx, dv, du, da);
    v and the half-step velocity move together."""
    def at(sign):
        q = oracle.copy_state(s)
        for c, k in enumerate("xyz"):
            q[k] = q[k] + sign * eps * dx[:, c]
            q["v" + k] = q["v" + k] + sign * eps * dv[:, c]
            q["v" + k + "h"] = q["v" + k + "h"] + sign * eps * dv[:, c]
        q["u"] = q["u"] + sign * eps * du
        return adj.frozen_loss(box, q, prm, tape, alpha=prm.alpha + sign * eps * da)[0]
    return (at(1.0) - at(-1.0)) / (2.0 * eps)


def _directions(n, rng, kind):
    z3, z1 = np.zeros((n, 3)), np.zeros(n)
    sx, sv, su = 1e-2 / 10, 0.05, 1.0        # spacing/10, velocity, internal energy scales
    if kind == "x":
        return rng.standard_normal((n, 3)) * sx, z3, z1, 0.0
    if kind == "v":
        return z3, rng.standard_normal((n, 3)) * sv, z1, 0.0
    if kind == "u":
        return z3, z3, rng.standard_normal(n) * su, 0.0
    if kind == "alpha":
        return z3, z3, z1, 1.0
    return (rng.standard_normal((n, 3)) * sx, rng.standard_normal((n, 3)) * sv,
            rng.standard_normal(n) * su, rng.standard_normal())


@pytest.mark.parametrize("kind", ["x", "v", "u", "alpha", "mixed", "mixed2"])
def test_reference_gradient_matches_central_differences(case, kind):
    s, box, prm, tape, g = case
    rng = np.random.default_rng(hash(kind) % 1000)
    dx, dv, du, da = _directions(s["x"].shape[0], rng, kind)
    fd = _fd(box, s, prm, tape, dx, dv, du, da, 1e-6)
    ad = (g["x"] * dx).sum() + (g["v"] * dv).sum() + (g["u"] * du).sum() + g["alpha"] * da
    # scale: the directional derivative with every term in magnitude
    scale = (np.abs(g["x"] * dx).sum() + np.abs(g["v"] * dv).sum() + np.abs(g["u"] * du).sum()
             + abs(g["alpha"] * da))
    assert abs(fd - ad) <= 1e-6 * scale, (fd, ad, scale)


def test_single_coordinates_match_central_differences(case):
    s, box, prm, tape, g = case
    n = s["x"].shape[0]
    rng = np.random.default_rng(5)
    for field in ("x", "v"):
        gf = g[field]
        for idx in rng.choice(n, 2, replace=False):
            for c in range(3):
                d3 = np.zeros((n, 3))
                d3[idx, c] = 1.0
                dx, dv = (d3, np.zeros((n, 3))) if field == "x" else (np.zeros((n, 3)), d3)
                fd = _fd(box, s, prm, tape, dx, dv, np.zeros(n), 0.0, 1e-6)
                assert abs(fd - gf[idx, c]) <= 1e-6 * np.abs(gf).max(), (field, idx, c)


def test_forward_mode_equals_reverse_mode(case):
    s, box, prm, tape, g = case
    rng = np.random.default_rng(11)
    for _ in range(2):
        dx, dv, du, da = _directions(s["x"].shape[0], rng, "mixed")
        jvp = adj.reference_jvp(box, s, prm, tape, dx, dv, du, da)
        vjp = (g["x"] * dx).sum() + (g["v"] * dv).sum() + (g["u"] * du).sum() + g["alpha"] * da
        assert jvp == pytest.approx(vjp, rel=1e-12)


def test_symmetry_closed_forms(case):
    s, box, prm, tape, g = case
    _, fin, _ = adj.frozen_loss(box, s, prm, tape)
    m = s["m"]
    # translation: sum_a dL/dx_a = 0
    assert np.abs(g["x"].sum(0)).max() <= 1e-12 * np.abs(g["x"]).sum()
    # Galilean shift: sum_a dL/dv_a = sum_a m_a v_a(K)
    pK = np.array([(m * fin["vx"]).sum(), (m * fin["vy"]).sum(), (m * fin["vz"]).sum()])
    np.testing.assert_allclose(g["v"].sum(0), pK, rtol=1e-10, atol=1e-13 * np.abs(g["v"]).sum())


@pytest.fixture(scope="module")
def case_gradh():
    s = sph_inputs.jittered_box(10, seed_index=72, vel_sigma=0.05)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    prm = oracle.Params(gradh=1)
    tape = adj.record(box, s, prm, 3)
    g = adj.reference_gradients(box, s, prm, tape)
    return s, box, prm, tape, g


def test_gradh_torch_forward_equals_c_oracle(case_gradh):
    s, box, prm, tape, _ = case_gradh
    L, fin, rho = adj.frozen_loss(box, s, prm, tape)
    x0, v0, u0, al = adj._inputs(s, prm.alpha)
    x, v, u, r = adj.torch_rollout(box, s, prm, tape, x0, v0, al, u0=u0)
    vr = np.stack([fin["vx"], fin["vy"], fin["vz"]], 1)
    assert np.abs(v.numpy() - vr).max() <= 1e-12 * np.abs(vr).max()
    np.testing.assert_allclose(r.numpy(), rho, rtol=1e-13)


@pytest.mark.parametrize("kind", ["x", "v", "mixed"])
def test_gradh_reference_gradient_matches_central_differences(case_gradh, kind):
    """With the grad-h terms the gradient also carries d Omega / dx (second
    derivatives of W), checked against central differences of the C oracle."""
    s, box, prm, tape, g = case_gradh
    rng = np.random.default_rng(hash(kind) % 1000 + 7)
    dx, dv, du, da = _directions(s["x"].shape[0], rng, kind)
    fd = _fd(box, s, prm, tape, dx, dv, du, da, 1e-6)
    ad = (g["x"] * dx).sum() + (g["v"] * dv).sum() + (g["u"] * du).sum() + g["alpha"] * da
    scale = (np.abs(g["x"] * dx).sum() + np.abs(g["v"] * dv).sum() + np.abs(g["u"] * du).sum()
             + abs(g["alpha"] * da))
    assert abs(fd - ad) <= 1e-6 * scale, (fd, ad, scale)
