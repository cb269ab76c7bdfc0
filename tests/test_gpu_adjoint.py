"""The differentiable rollout (hand-written adjoint kernels, checkpointing):
gradients of L = sum (rho - 1)^2 + sum m |v|^2 / 2 after K FP64 steps with
respect to the initial positions, velocities, internal energies and alpha,
with neighbour lists, h, dt and the viscosity switch held at their forward
values.

Checked against (a) the reference adjoint (reverse-mode AD of the oracle's
PyTorch restatement, itself pinned to the C oracle and to central
differences on the CPU), (b) central differences of the C oracle's frozen
rollout, (c) invariance of the result under the checkpoint interval and
repetition, and (d) at 10^6 particles the symmetry closed forms
sum_a dL/dx_a = 0 and sum_a dL/dv_a = sum_a m_a v_a(K).

Tolerance: the gradients are exact derivatives of the same function on both
sides, so they differ by FP64 rounding of the pair sums amplified through K
steps.  "Relative 1e-6" is read per field as max |g - g_ref| <= 1e-6
max |g_ref| (a component that is zero by symmetry has no relative error),
and in addition per component, |g_i - g_ref,i| <= 1e-6 |g_ref,i|, for every
component at least 1e-4 of the field's largest; against central differences
it is 1e-6 of the directional derivative with every term in magnitude.
Measured differences are far below these bars."""
import numpy as np
import pytest
import torch

import oracle
import sph_inputs
from oracle import adjoint as adj

pytestmark = pytest.mark.gpu

K, EVERY = 20, 5
TOL = 1e-6


def _case(side=10, seed=70, vel=0.05):
    s = sph_inputs.jittered_box(side, seed_index=seed, vel_sigma=vel)
    return s, oracle.Box(s["lo"], s["hi"], s["periodic"])


def _gpu_grad(s, steps=K, every=EVERY, alpha=1.0, ro=None, return_final=False):
    from paper_2005_02656_gb300 import Params, Rollout
    n = s["x"].shape[0]
    own = ro is None
    if own:
        ro = Rollout(n, steps, every, Params(box_lo=s["lo"], box_hi=s["hi"],
                                             periodic=s["periodic"]))
    dev = ro.device
    st = {k: torch.as_tensor(s[k], dtype=torch.float64, device=dev)
          for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u", "du_prev")}
    fin = ro.forward(st, alpha)
    m = st["m"]
    g = torch.zeros_like(fin)
    g[3:6] = m[None, :] * fin[3:6]                 # d/dv of sum m |v|^2 / 2
    g[7] = 2.0 * (fin[7] - 1.0)                    # d/drho of sum (rho - 1)^2
    gi, ga = ro.backward(g)
    torch.cuda.synchronize()
    gi = gi.cpu().numpy()
    out = {"x": gi[0:3].T.copy(), "v": (gi[3:6] + gi[6:9]).T.copy(), "u": gi[9].copy(),
           "vh": gi[6:9].T.copy(), "du_prev": gi[10].copy(), "alpha": float(ga.cpu()),
           "dt": ro.time_steps(), "info": ro.info()}
    f = fin.cpu().numpy()
    out["loss"] = adj.loss_of(f[7], f[3:6].T, s["m"])
    if return_final:
        out["final"] = f
    if own:
        ro.close()
    return out


@pytest.fixture(scope="module")
def small():
    s, box = _case()
    prm = oracle.Params()
    tape = adj.record(box, s, prm, K)
    ref = adj.reference_gradients(box, s, prm, tape)
    gpu = _gpu_grad(s)
    return s, box, prm, tape, ref, gpu


def test_forward_matches_oracle_and_time_steps(small):
    s, box, prm, tape, ref, gpu = small
    np.testing.assert_allclose(gpu["dt"], np.array(tape.dt), rtol=1e-12)
    assert gpu["loss"] == pytest.approx(ref["loss"], rel=1e-10)


@pytest.mark.parametrize("field", ["x", "v", "u"])
def test_gradient_matches_reference_adjoint(small, field):
    *_, ref, gpu = small
    g, r = np.asarray(gpu[field]), np.asarray(ref[field])
    err = np.abs(g - r).max()
    assert err <= TOL * np.abs(r).max(), (field, err, np.abs(r).max())
    # component by component where the component is not tiny
    big = np.abs(r) >= 1e-4 * np.abs(r).max()
    assert big.sum() > 0.5 * big.size
    rel = np.abs(g - r)[big] / np.abs(r)[big]
    assert rel.max() <= TOL, (field, rel.max())


def test_alpha_gradient_matches_reference_adjoint(small):
    *_, ref, gpu = small
    assert gpu["alpha"] == pytest.approx(ref["alpha"], rel=TOL)


def test_gradient_matches_central_differences(small):
    """32 random directions (x, v, u and alpha together) and 16 single
    coordinates, central differences of the C oracle's frozen rollout."""
    s, box, prm, tape, _, gpu = small
    n = s["x"].shape[0]
    rng = np.random.default_rng(2005)
    sx, sv, su = 1e-2 / 10, 0.05, 1.0

    def fd(dx, dv, du, da, eps):
        def at(sign):
            q = oracle.copy_state(s)
            for c, k in enumerate("xyz"):
                q[k] = q[k] + sign * eps * dx[:, c]
                q["v" + k] = q["v" + k] + sign * eps * dv[:, c]
                q["v" + k + "h"] = q["v" + k + "h"] + sign * eps * dv[:, c]
            q["u"] = q["u"] + sign * eps * du
            return adj.frozen_loss(box, q, prm, tape, alpha=prm.alpha + sign * eps * da)[0]
        return (at(1.0) - at(-1.0)) / (2.0 * eps)

    worst = 0.0
    for _ in range(32):
        dx = rng.standard_normal((n, 3)) * sx
        dv = rng.standard_normal((n, 3)) * sv
        du = rng.standard_normal(n) * su
        da = rng.standard_normal()
        ad = (gpu["x"] * dx).sum() + (gpu["v"] * dv).sum() + (gpu["u"] * du).sum() + gpu["alpha"] * da
        scale = (np.abs(gpu["x"] * dx).sum() + np.abs(gpu["v"] * dv).sum()
                 + np.abs(gpu["u"] * du).sum() + abs(gpu["alpha"] * da))
        worst = max(worst, abs(fd(dx, dv, du, da, 1e-6) - ad) / scale)
    assert worst <= TOL, worst
    # single coordinates: a step of 1e-6 in absolute units (1e-5 of the
    # spacing; 2e-5 of the velocity scale) keeps the rounding of L (~1e-16)
    # well below the change of L it measures
    z3, z1 = np.zeros((n, 3)), np.zeros(n)
    for t in range(16):
        i, c = int(rng.integers(n)), int(rng.integers(3))
        d3 = np.zeros((n, 3))
        d3[i, c] = 1.0
        if t % 2 == 0:
            got, exp = gpu["x"][i, c], fd(d3, z3, z1, 0.0, 1e-6)
            scale = np.abs(gpu["x"]).max()
        else:
            got, exp = gpu["v"][i, c], fd(z3, d3, z1, 0.0, 1e-6)
            scale = np.abs(gpu["v"]).max()
        assert abs(got - exp) <= TOL * scale, (t, i, c, got, exp)


def test_checkpoint_interval_and_repetition_are_bit_exact(small):
    """Recomputing segments from checkpoints reproduces the forward exactly,
    and every reverse sum runs in a fixed order."""
    from paper_2005_02656_gb300 import Params, Rollout
    s, *_, gpu = small
    assert gpu["info"]["recomputed_steps"] == K - EVERY
    for every in (1, 7, K):
        other = _gpu_grad(s, every=every)
        for k in ("x", "v", "u", "vh", "du_prev"):
            np.testing.assert_array_equal(other[k], gpu[k], err_msg=f"every={every} {k}")
        assert other["alpha"] == gpu["alpha"]
    n = s["x"].shape[0]
    ro = Rollout(n, K, EVERY, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"]))
    a = _gpu_grad(s, ro=ro)
    b = _gpu_grad(s, ro=ro)                      # second forward + backward on one context
    for k in ("x", "v", "u"):
        np.testing.assert_array_equal(a[k], b[k])
    ro.close()


def test_autograd_function_gives_the_same_gradients(small):
    from paper_2005_02656_gb300 import Params, Rollout, rollout
    s, *_, gpu = small
    n = s["x"].shape[0]
    dev = torch.device("cuda:0")
    ro = Rollout(n, K, EVERY, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"]))
    x0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1), device=dev, requires_grad=True)
    v0 = torch.tensor(np.stack([s["vx"], s["vy"], s["vz"]], 1), device=dev, requires_grad=True)
    u0 = torch.tensor(s["u"], device=dev, requires_grad=True)
    alpha = torch.tensor(1.0, dtype=torch.float64, device=dev, requires_grad=True)
    h = torch.tensor(s["h"], device=dev)
    m = torch.tensor(s["m"], device=dev)
    x, v, u, rho = rollout(x0, v0, u0, alpha, ro, h, m)
    loss = ((rho - 1.0) ** 2).sum() + 0.5 * (m * (v * v).sum(1)).sum()
    loss.backward()
    np.testing.assert_allclose(x0.grad.cpu().numpy(), gpu["x"], rtol=0,
                               atol=1e-12 * np.abs(gpu["x"]).max())
    np.testing.assert_allclose(v0.grad.cpu().numpy(), gpu["v"], rtol=0,
                               atol=1e-12 * np.abs(gpu["v"]).max())
    np.testing.assert_allclose(u0.grad.cpu().numpy(), gpu["u"], rtol=0,
                               atol=1e-12 * np.abs(gpu["u"]).max())
    assert float(alpha.grad) == pytest.approx(gpu["alpha"], rel=1e-12)
    ro.close()


def test_stale_graph_backward_is_refused():
    """A Rollout keeps the tape of its last forward only: the backward of an
    earlier graph after a newer forward on the same Rollout raises instead of
    returning the newer rollout's gradients."""
    from paper_2005_02656_gb300 import Params, Rollout, rollout
    s, _ = _case(side=8, seed=72)
    n = s["x"].shape[0]
    dev = torch.device("cuda:0")
    ro = Rollout(n, 2, 1, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"]))
    h = torch.tensor(s["h"], device=dev)
    m = torch.tensor(s["m"], device=dev)

    def run(scale):
        x0 = torch.tensor(np.stack([s["x"], s["y"], s["z"]], 1), device=dev, requires_grad=True)
        v0 = torch.tensor(scale * np.stack([s["vx"], s["vy"], s["vz"]], 1), device=dev,
                          requires_grad=True)
        u0 = torch.tensor(s["u"], device=dev, requires_grad=True)
        x, v, u, rho = rollout(x0, v0, u0, 1.0, ro, h, m)
        return ((rho - 1.0) ** 2).sum() + 0.5 * (m * (v * v).sum(1)).sum()

    first = run(1.0)
    second = run(2.0)
    with pytest.raises(RuntimeError, match="another forward"):
        first.backward()
    second.backward()                     # the newest graph still differentiates
    ro.close()


def test_backward_before_forward_and_overflow_are_errors():
    from paper_2005_02656_gb300 import Params, Rollout, _lib
    s, _ = _case(side=8, seed=71)
    n = s["x"].shape[0]
    ro = Rollout(n, 2, 1, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"]))
    with pytest.raises(_lib.SphError) as e:
        ro.backward(torch.zeros(8, n, dtype=torch.float64, device="cuda:0"))
    assert e.value.code == _lib.SPH_ERR_ORDER
    ro.close()
    ro = Rollout(n, 2, 1, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                                 max_nb=32))
    with pytest.raises(_lib.SphError) as e:
        _gpu_grad(s, steps=2, every=1, ro=ro)
    assert e.value.code == _lib.SPH_ERR_NB_OVERFLOW
    ro.close()


def test_full_size_symmetry_closed_forms():
    """10^6 particles (100^3 jittered periodic box), K = 20, checkpoint every
    5: translation and Galilean closed forms of the gradient."""
    s, _ = _case(side=100, seed=3, vel=0.01)
    g = _gpu_grad(s, return_final=True)
    for k in ("x", "v", "u"):
        assert np.isfinite(g[k]).all()
    assert np.isfinite(g["alpha"])
    assert np.abs(g["x"].sum(0)).max() <= 1e-10 * np.abs(g["x"]).sum()
    f = g["final"]
    pK = (s["m"][None, :] * f[3:6]).sum(1)
    assert np.abs(g["v"].sum(0) - pK).max() <= 1e-10 * (np.abs(g["v"]).sum() + np.abs(pK).sum())
    assert g["info"]["recomputed_steps"] == K - EVERY


def test_gradh_adjoint_matches_reference_and_central_differences():
    """With the grad-h terms (gradh = 1) the reverse pass also carries
    dOmega/dx (second derivatives of W): against the reference adjoint with
    the same Omega and against central differences of the C oracle."""
    from paper_2005_02656_gb300 import Params, Rollout
    s, box = _case(side=10, seed=73)
    prm = oracle.Params(gradh=1)
    steps = 6
    tape = adj.record(box, s, prm, steps)
    ref = adj.reference_gradients(box, s, prm, tape)
    n = s["x"].shape[0]
    ro = Rollout(n, steps, 3, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                                     gradh=1))
    gpu = _gpu_grad(s, steps=steps, every=3, ro=ro)
    ro.close()
    np.testing.assert_allclose(gpu["dt"], np.array(tape.dt), rtol=1e-12)
    for field in ("x", "v", "u"):
        err = np.abs(gpu[field] - ref[field]).max()
        assert err <= TOL * np.abs(ref[field]).max(), (field, err)
    assert gpu["alpha"] == pytest.approx(ref["alpha"], rel=TOL)
    rng = np.random.default_rng(17)
    sx, sv = 1e-3, 0.05
    for _ in range(4):
        dx = rng.standard_normal((n, 3)) * sx
        dv = rng.standard_normal((n, 3)) * sv

        def at(sign):
            q = oracle.copy_state(s)
            for c, k in enumerate("xyz"):
                q[k] = q[k] + sign * 1e-6 * dx[:, c]
                q["v" + k] = q["v" + k] + sign * 1e-6 * dv[:, c]
                q["v" + k + "h"] = q["v" + k + "h"] + sign * 1e-6 * dv[:, c]
            return adj.frozen_loss(box, q, prm, tape)[0]
        fd = (at(1.0) - at(-1.0)) / 2e-6
        ad = (gpu["x"] * dx).sum() + (gpu["v"] * dv).sum()
        scale = np.abs(gpu["x"] * dx).sum() + np.abs(gpu["v"] * dv).sum()
        assert abs(fd - ad) <= TOL * scale, (fd, ad)
