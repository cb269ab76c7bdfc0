"""Reference adjoint of K SPH steps with frozen neighbour lists, smoothing
lengths and time steps (test infrastructure only).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's CPU
baseline use this module; the product path never does.  It imports nothing
from the product.

What is differentiated.  A rollout of K steps of the method of section 4.1
(Eq. 1 density with the self term, the ideal-gas EOS, the IAD matrix
C = tau^{-1}, Eqs. 2-5 momentum and energy with artificial viscosity, the
leapfrog / Adams-Bashforth update with the readings stated in
``sph_oracle.c``), followed by one density pass on the final state, and the
scalar

    L = sum_a (rho_a - 1)^2 + sum_a m_a |v_a|^2 / 2

of the final density and velocities.  The neighbour lists of every step (and
of the final density pass), the smoothing lengths, the time steps and the
viscosity switch of Eq. 5 (on where x_ab . v_ab < 0) are held at the values
of a base run.  The lists, h and the switch are piecewise constant in the
inputs and dt is a minimum, so the frozen rollout is the smooth function whose
gradient an adjoint computes; at the base point its derivative is the
rollout's own.  (Without the frozen switch, central differences at K = 20 on
a 10^3 box cross the switch's kink for about one pair in a million pair-steps
and miss the derivative by ~1e-5.)

Three pieces, each independent of the others' arithmetic:
  * ``record``        a base run of the C oracle that stores, per step, the
                      lists, h, dt, dt_prev and the viscosity switch;
  * ``frozen_loss``   the same rollout through the C oracle's own functions
                      with the recorded lists, time steps and switch: the
                      function that central finite differences are taken of;
  * ``torch_rollout`` a plain PyTorch FP64 restatement of the same equations
                      over per-pair index arrays, whose reverse-mode
                      derivative (``reference_gradients``) and forward-mode
                      dual-number derivative (``reference_jvp``) are the
                      reference adjoint.
The torch restatement is pinned to the C oracle by equal forward values, and
its derivatives to central differences of ``frozen_loss``.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import (OK, Box, Params, copy_state, density_eos, find_neighbors, iad, kernel_norm,
               momentum_energy, update)


@dataclass
class Tape:
    """Per-step frozen quantities of a base run (index order of the inputs)."""
    nn: list          # per step: int32 (n,) true neighbour counts
    nbr: list         # per step: int64 (n, max_nb) sorted lists, -1 padded
    dt: list          # per step: the time step used
    dt_prev: list     # per step: the previous time step (0 on the first)
    h: list           # per step: smoothing lengths used by that step
    av: list          # per step: int8 viscosity switch per list entry
    nn_final: np.ndarray
    nbr_final: np.ndarray
    h_final: np.ndarray


def loss_of(rho, v, m):
    """L = sum (rho - 1)^2 + sum m |v|^2 / 2 (numpy, compensated sums)."""
    return math.fsum(((rho - 1.0) ** 2).tolist()) + math.fsum((0.5 * m * (v ** 2).sum(1)).tolist())


def record(box: Box, s0: dict, params: Params, steps: int, dt_prev0: float = 0.0) -> Tape:
    """Base run of ``steps`` full oracle steps from ``s0`` (not modified)."""
    from . import step as oracle_step
    s = copy_state(s0)
    tape = Tape([], [], [], [], [], [], None, None, None)
    dt_prev = dt_prev0
    for _ in range(steps):
        tape.h.append(s["h"].copy())
        rc, dt, out = oracle_step(box, s, params, dt_prev, record_av=True)
        if rc != OK:
            raise RuntimeError(f"oracle step failed: {rc}")
        tape.av.append(out["av"])
        tape.nn.append(out["nn"].copy())
        tape.nbr.append(out["nbr"].copy())
        tape.dt.append(dt)
        tape.dt_prev.append(dt_prev)
        dt_prev = dt
    rc, nn, nbr = find_neighbors(box, s["x"], s["y"], s["z"], s["h"], max_nb=params.max_nb)
    if rc != OK:
        raise RuntimeError(f"oracle neighbour search failed: {rc}")
    tape.nn_final, tape.nbr_final, tape.h_final = nn, nbr, s["h"].copy()
    return tape


def frozen_loss(box: Box, s0: dict, params: Params, tape: Tape, alpha: float | None = None):
    """L of the rollout with the tape's lists and time steps, evaluated with
    the C oracle's functions.  Returns (L, final state, final rho)."""
    prm = Params(**{**params.__dict__})
    if alpha is not None:
        prm.alpha = float(alpha)
    Bn = kernel_norm(prm.sinc_n)
    s = copy_state(s0)
    for k in range(len(tape.dt)):
        nn, nbr = tape.nn[k], tape.nbr[k]
        omega = None
        if prm.gradh:
            rho, p, c, omega = density_eos(box, s, nn, nbr, prm, Bn=Bn, with_omega=True)
        else:
            rho, p, c = density_eos(box, s, nn, nbr, prm, Bn=Bn)
        _, C6, _ = iad(box, s, rho, nn, nbr, prm, Bn=Bn)
        me = momentum_energy(box, s, rho, p, c, C6, nn, nbr, prm, Bn=Bn, av_force=tape.av[k],
                             omega_full=omega)
        update(box, s, me["ax"], me["ay"], me["az"], me["du"], nn, tape.dt[k], tape.dt_prev[k],
               prm.ng_target)
    rho, _, _ = density_eos(box, s, tape.nn_final, tape.nbr_final, prm, Bn=Bn)
    v = np.stack([s["vx"], s["vy"], s["vz"]], 1)
    return loss_of(rho, v, s["m"]), s, rho


# ---------------------------------------------------------------------------
# PyTorch FP64 restatement (CPU).  Pairs are (a, b) with b in the list of a;
# every per-pair quantity is a 1-D tensor over pairs and sums over b are
# index_add over a.
# ---------------------------------------------------------------------------

def _pairs(nbr: np.ndarray, av: np.ndarray | None = None):
    a, k = np.nonzero(nbr >= 0)
    out = (torch.as_tensor(a, dtype=torch.int64), torch.as_tensor(nbr[a, k], dtype=torch.int64))
    if av is None:
        return out
    return out + (torch.as_tensor(av[a, k] != 0),)


def _sep(box: Box, x, a, b):
    """x_b - x_a per pair with the minimum image on periodic axes (n, 3) -> (P, 3)."""
    d = x[b] - x[a]
    cols = []
    for k in range(3):
        dk = d[:, k]
        if box.periodic[k]:
            L = float(box.hi[k]) - float(box.lo[k])
            dk = torch.where(dk > 0.5 * L, dk - L, torch.where(dk < -0.5 * L, dk + L, dk))
        cols.append(dk)
    return torch.stack(cols, 1)


def _W(v, h, Bn: float, sinc_n: float):
    """Eq. 6: B_n / h^3 [sin(pi v/2) / (pi v/2)]^n for 0 < v <= 2."""
    xq = 0.5 * math.pi * v
    return Bn / h ** 3 * (torch.sin(xq) / xq) ** sinc_n


def _dWdh(v, h, Bn: float, sinc_n: float):
    """dW/dh at fixed separation: -(3 W + v dW/dv) / h, with
    dW/dv = B_n / h^3 n S^(n-1) (pi/2) (x cos x - sin x) / x^2, x = pi v / 2."""
    xq = 0.5 * math.pi * v
    S = torch.sin(xq) / xq
    dS = 0.5 * math.pi * (xq * torch.cos(xq) - torch.sin(xq)) / (xq * xq)
    W = Bn / h ** 3 * S ** sinc_n
    dWdv = Bn / h ** 3 * sinc_n * S ** (sinc_n - 1.0) * dS
    return -(3.0 * W + v * dWdv) / h


def _density(box, x, h, m, u, a, b, Bn, prm, with_omega=False):
    """Eq. 1 with the self term and the EOS; with_omega also returns the
    grad-h terms Omega = 1 + h / (3 rho) sum_b m_b dW/dh (self term included)."""
    d = _sep(box, x, a, b)
    r = torch.sqrt((d * d).sum(1))
    rho = m * Bn / h ** 3                    # self term, W(0, h) = B_n / h^3
    rho = rho.index_add(0, a, m[b] * _W(r / h[a], h[a], Bn, prm.sinc_n))
    p = (prm.gamma - 1.0) * rho * u
    c = torch.sqrt(prm.gamma * p / rho)
    if not with_omega:
        return rho, p, c, d, r
    dsum = m * (-3.0 * Bn / h ** 4)          # self term: dW(0, h)/dh = -3 B_n / h^4
    dsum = dsum.index_add(0, a, m[b] * _dWdh(r / h[a], h[a], Bn, prm.sinc_n))
    omega = 1.0 + h / (3.0 * rho) * dsum
    return rho, p, c, d, r, omega


def _step(box, st, h, m, nn, nbr, av, dt, dt_prev, alpha, Bn, prm):
    x, v, vh, u, du_prev = st
    a, b, on = _pairs(nbr, av)
    if prm.gradh:
        rho, p, c, d, r, omega = _density(box, x, h, m, u, a, b, Bn, prm, with_omega=True)
    else:
        rho, p, c, d, r = _density(box, x, h, m, u, a, b, Bn, prm)
        omega = torch.ones_like(rho)
    # IAD: tau_a = sum_b (m_b / rho_b) W_ab(h_a) d d^T, C_a = tau_a^{-1}
    Wa = _W(r / h[a], h[a], Bn, prm.sinc_n)
    w = (m[b] / rho[b] * Wa)[:, None, None] * d[:, :, None] * d[:, None, :]
    tau = torch.zeros(x.shape[0], 3, 3, dtype=x.dtype).index_add(0, a, w)
    C = torch.linalg.inv(tau)
    # Eqs. 2-5
    va = (r / h[b])
    Wb = torch.where(va < 2.0, _W(torch.clamp(va, max=2.0), h[b], Bn, prm.sinc_n),
                     torch.zeros_like(va))
    Aa = torch.einsum("pij,pj->pi", C[a], d) * Wa[:, None]
    Ab = torch.einsum("pij,pj->pi", C[b], d) * Wb[:, None]
    X = p / (omega * rho ** 2)              # P / (Omega rho^2), Eqs. 2-3
    Xa, Xb = X[a], X[b]
    vab = v[a] - v[b]
    xv = (-d * vab).sum(1)
    wv = xv / r
    vsig = c[a] + c[b] - 3.0 * wv
    Pi = torch.where(on, -0.5 * alpha * vsig * wv, torch.zeros_like(xv))
    Abar = Aa / rho[a][:, None] + Ab / rho[b][:, None]
    term = -m[b][:, None] * (Xa[:, None] * Aa + Xb[:, None] * Ab) \
        - 0.5 * m[b][:, None] * Pi[:, None] * Abar
    eterm = Xa * m[b] * (vab * Aa).sum(1) + 0.25 * m[b] * Pi * (vab * Abar).sum(1)
    acc = torch.zeros_like(x).index_add(0, a, term)
    du = torch.zeros_like(u).index_add(0, a, eterm)
    # update (readings stated in sph_oracle.c), dt and dt_prev frozen
    delta = 0.5 * (dt + dt_prev)
    vh = vh + acc * delta
    xn = x + dt * vh
    cols = []
    for k in range(3):
        xk = xn[:, k]
        if box.periodic[k]:
            lo, hi = float(box.lo[k]), float(box.hi[k])
            xk = torch.where(xk >= hi, xk - (hi - lo), torch.where(xk < lo, xk + (hi - lo), xk))
        cols.append(xk)
    xn = torch.stack(cols, 1)
    vn = vh + 0.5 * dt * acc
    if dt_prev > 0.0:
        q = dt / (2.0 * dt_prev)
        un = u + dt * ((1.0 + q) * du - q * du_prev)
    else:
        un = u + dt * du
    return (xn, vn, vh, un, du)


def torch_rollout(box: Box, s0: dict, params: Params, tape: Tape, x0, v0, alpha, u0=None,
                  vh0=None):
    """Final (x, v, u, rho) of the frozen rollout, as functions of the tensors
    x0 (n, 3), v0 (n, 3), alpha (0-d), u0 (n) and vh0 (n, 3; defaults to v0)."""
    Bn = kernel_norm(params.sinc_n)
    m = torch.as_tensor(s0["m"], dtype=torch.float64)
    if u0 is None:
        u0 = torch.as_tensor(s0["u"], dtype=torch.float64)
    du_prev = torch.as_tensor(s0["du_prev"], dtype=torch.float64)
    st = (x0, v0, v0 if vh0 is None else vh0, u0, du_prev)
    for k in range(len(tape.dt)):
        h = torch.as_tensor(tape.h[k], dtype=torch.float64)
        st = _step(box, st, h, m, tape.nn[k], tape.nbr[k], tape.av[k], tape.dt[k],
                   tape.dt_prev[k], alpha, Bn, params)
    x, v, _, u, _ = st
    a, b = _pairs(tape.nbr_final)
    h = torch.as_tensor(tape.h_final, dtype=torch.float64)
    rho, _, _, _, _ = _density(box, x, h, m, u, a, b, Bn, params)
    return x, v, u, rho


def torch_loss(rho, v, m):
    return ((rho - 1.0) ** 2).sum() + (0.5 * m * (v * v).sum(1)).sum()


def _inputs(s0, alpha):
    x0 = torch.as_tensor(np.stack([s0["x"], s0["y"], s0["z"]], 1), dtype=torch.float64)
    v0 = torch.as_tensor(np.stack([s0["vx"], s0["vy"], s0["vz"]], 1), dtype=torch.float64)
    u0 = torch.as_tensor(s0["u"], dtype=torch.float64)
    al = torch.tensor(float(alpha), dtype=torch.float64)
    return x0, v0, u0, al


def reference_gradients(box: Box, s0: dict, params: Params, tape: Tape, alpha=None):
    """dL/dx0 (n, 3), dL/dv0 (n, 3; v0 also seeds the half-step velocity),
    dL/du0 (n) and dL/dalpha by reverse-mode AD of ``torch_rollout``."""
    alpha = params.alpha if alpha is None else alpha
    x0, v0, u0, al = _inputs(s0, alpha)
    for t in (x0, v0, u0, al):
        t.requires_grad_(True)
    x, v, u, rho = torch_rollout(box, s0, params, tape, x0, v0, al, u0=u0)
    m = torch.as_tensor(s0["m"], dtype=torch.float64)
    L = torch_loss(rho, v, m)
    gx, gv, gu, ga = torch.autograd.grad(L, (x0, v0, u0, al))
    return {"loss": float(L.detach()), "x": gx.numpy(), "v": gv.numpy(), "u": gu.numpy(),
            "alpha": float(ga)}


def reference_jvp(box: Box, s0: dict, params: Params, tape: Tape, dx, dv, du, dalpha, alpha=None):
    """Directional derivative of L along (dx, dv, du, dalpha) by forward-mode
    (dual-number) AD of ``torch_rollout``."""
    import torch.autograd.forward_ad as fwAD
    alpha = params.alpha if alpha is None else alpha
    x0, v0, u0, al = _inputs(s0, alpha)
    m = torch.as_tensor(s0["m"], dtype=torch.float64)
    with fwAD.dual_level():
        xd = fwAD.make_dual(x0, torch.as_tensor(dx, dtype=torch.float64))
        vd = fwAD.make_dual(v0, torch.as_tensor(dv, dtype=torch.float64))
        ud = fwAD.make_dual(u0, torch.as_tensor(du, dtype=torch.float64))
        ad = fwAD.make_dual(al, torch.tensor(float(dalpha), dtype=torch.float64))
        x, v, u, rho = torch_rollout(box, s0, params, tape, xd, vd, ad, u0=ud)
        L = torch_loss(rho, v, m)
        return float(fwAD.unpack_dual(L).tangent)
