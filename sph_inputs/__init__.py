"""Seeded synthetic SPH initial conditions (shared by the tests, the smoke check
and the benchmark).

This module holds only the workload recipes: lattices, jitter, masses,
velocities, internal energy and the initial smoothing length.  It holds none of
the method's arithmetic (no kernel, sums, EOS or integrator).  Every generator
is seeded with numpy's PCG64 at ``SEED_BASE + workload index``.

A state is a dict of FP64 numpy arrays with the keys
``x y z vx vy vz vxh vyh vzh h m u du_prev`` plus ``id`` (int64), and the
box as ``lo``, ``hi`` (3-tuples) and ``periodic`` (3-tuple of 0/1).  ``vxh``
etc. start equal to ``v`` and ``du_prev`` at zero: the integrator's state
before the first step.

Workloads (the paper's setups, section 4.6 and the configurations measured):
  * ``jittered_box``   periodic unit box, cubic lattice jittered by U(-0.1, 0.1)
                       spacing per axis, m = 1/N, u = 1, v ~ N(0, 0.01^2).
  * ``square_patch``   section 4.6: 3-D rotating square patch, lattice on
                       [-0.5, 0.5]^3, x and y open, z periodic, density 1,
                       u = 1, v = (omega y, -omega x, 0), omega = 5 (Eq. 7).
  * ``kelvin_helmholtz`` periodic [0,1] x [0,1] x [0,0.5] shear layer: density
                       2 for 0.25 <= y < 0.75 and 1 elsewhere with equal-mass
                       particles from two cubic lattices, vx = +0.5 inside and
                       -0.5 outside, vy = 0.01 sin(4 pi x), pressure 2.5 with
                       gamma = 5/3 (u = 3.75 / rho).
  * ``ensemble``       boxes of the jittered-box recipe, side counts drawn
                       log-uniformly from [8, 48], alpha uniform in [0.5, 1.5].
  * ``uniform_sphere`` the self-gravity workload: the lattice points of
                       [-1, 1]^3 inside the unit sphere, jittered by U(-0.1,
                       0.1) spacing, total mass 1, at rest, u = 1, open
                       boundaries.
"""
from __future__ import annotations

import math

import numpy as np

SEED_BASE = 200502656
NG_TARGET = 100


def h_for_neighbors(spacing: float, ng: int = NG_TARGET) -> float:
    """Smoothing length whose 2h sphere holds ``ng`` particles at lattice spacing
    ``spacing`` (mean-density count): (4/3) pi (2h)^3 = ng spacing^3."""
    return spacing * (3.0 * ng / (4.0 * math.pi)) ** (1.0 / 3.0) / 2.0


def _lattice(nx: int, ny: int, nz: int, lo, spacing):
    sx, sy, sz = spacing if np.ndim(spacing) else (spacing,) * 3
    i = (np.arange(nx) + 0.5) * sx + lo[0]
    j = (np.arange(ny) + 0.5) * sy + lo[1]
    k = (np.arange(nz) + 0.5) * sz + lo[2]
    Z, Y, X = np.meshgrid(k, j, i, indexing="ij")
    return X.ravel().copy(), Y.ravel().copy(), Z.ravel().copy()


def _finish(x, y, z, vx, vy, vz, h, m, u, lo, hi, periodic, rng=None, shuffle=True):
    n = x.shape[0]
    ids = np.arange(n, dtype=np.int64)
    if shuffle:
        # present the particles in a random order: the library must sort them
        g = rng if rng is not None else np.random.default_rng(SEED_BASE)
        perm = g.permutation(n)
        x, y, z, vx, vy, vz, h, m, u, ids = (a[perm] for a in (x, y, z, vx, vy, vz, h, m, u, ids))
    s = {
        "x": x, "y": y, "z": z, "vx": vx, "vy": vy, "vz": vz,
        "vxh": vx.copy(), "vyh": vy.copy(), "vzh": vz.copy(),
        "h": h, "m": m, "u": u, "du_prev": np.zeros(n), "id": ids,
        "lo": tuple(float(a) for a in lo), "hi": tuple(float(a) for a in hi),
        "periodic": tuple(int(p) for p in periodic),
    }
    for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u", "du_prev"):
        s[k] = np.ascontiguousarray(s[k], dtype=np.float64)
    return s


def jittered_box(side: int = 20, seed_index: int = 0, jitter: float = 0.1, vel_sigma: float = 0.01,
                 u0: float = 1.0, ng: int = NG_TARGET, length: float = 1.0, shuffle=True):
    """Periodic cube of ``side^3`` particles: lattice at (i + 1/2) spacing,
    jittered uniformly by +-``jitter`` spacing per axis, m = 1/N (density 1 for
    the unit box), u = ``u0``, Gaussian velocities of std ``vel_sigma``."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    dx = length / side
    x, y, z = _lattice(side, side, side, (0.0, 0.0, 0.0), dx)
    n = x.shape[0]
    x = x + rng.uniform(-jitter, jitter, n) * dx
    y = y + rng.uniform(-jitter, jitter, n) * dx
    z = z + rng.uniform(-jitter, jitter, n) * dx
    v = rng.normal(0.0, vel_sigma, (3, n))
    h = np.full(n, h_for_neighbors(dx, ng))
    m = np.full(n, length ** 3 / n)
    u = np.full(n, u0)
    return _finish(x, y, z, v[0], v[1], v[2], h, m, u, (0.0, 0.0, 0.0), (length,) * 3, (1, 1, 1),
                   rng=rng, shuffle=shuffle)


def square_patch(side: int = 100, omega: float = 5.0, seed_index: int = 1, ng: int = NG_TARGET,
                 shuffle=True):
    """Section 4.6 rotating square patch in 3-D: ``side^3`` lattice on
    [-0.5, 0.5]^3, x and y open, z periodic (length 1), density 1, u = 1,
    rigid rotation v = (omega y, -omega x, 0) (Eq. 7)."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    dx = 1.0 / side
    x, y, z = _lattice(side, side, side, (-0.5, -0.5, -0.5), dx)
    n = x.shape[0]
    vx = omega * y
    vy = -omega * x
    vz = np.zeros(n)
    h = np.full(n, h_for_neighbors(dx, ng))
    m = np.full(n, 1.0 / n)
    u = np.ones(n)
    return _finish(x, y, z, vx, vy, vz, h, m, u, (-0.5, -0.5, -0.5), (0.5, 0.5, 0.5), (0, 0, 1),
                   rng=rng, shuffle=shuffle)


def kelvin_helmholtz(nx_outer: int = 224, seed_index: int = 2, ng: int = NG_TARGET, shuffle=True,
                     pressure: float = 2.5, gamma: float = 5.0 / 3.0):
    """Shear layer in the periodic box [0,1] x [0,1] x [0,0.5].

    Outer region (y < 0.25 or y >= 0.75, contiguous through the periodic y
    boundary): cubic lattice of spacing 1/nx_outer, density 1.  Inner region
    (0.25 <= y < 0.75): cubic lattice of spacing 1/nx_inner with
    nx_inner = the even integer nearest nx_outer * 2^(1/3), density 2, so that
    particle masses agree to a fraction of a percent.  nx_outer = 224 gives
    224x112x112 + 282x141x141 = 8,416,298 particles.  vx = +0.5 inside and
    -0.5 outside, vy = 0.01 sin(4 pi x), vz = 0, uniform pressure 2.5
    (u = P / ((gamma - 1) rho)), h set for ``ng`` neighbours per region."""
    if nx_outer % 4:
        raise ValueError("nx_outer must be a multiple of 4")
    rng = np.random.default_rng(SEED_BASE + seed_index)
    no = nx_outer
    ni = 2 * int(round(no * 2.0 ** (1.0 / 3.0) / 2.0))
    do, di = 1.0 / no, 1.0 / ni
    # outer: two slabs of no/4 layers each in y, no layers in x, no/2 in z
    xo1, yo1, zo1 = _lattice(no, no // 4, no // 2, (0.0, 0.0, 0.0), do)
    xo2, yo2, zo2 = _lattice(no, no // 4, no // 2, (0.0, 0.75, 0.0), do)
    xi, yi, zi = _lattice(ni, ni // 2, ni // 2, (0.0, 0.25, 0.0), di)
    xo, yo, zo = (np.concatenate(p) for p in ((xo1, xo2), (yo1, yo2), (zo1, zo2)))
    n_o, n_i = xo.shape[0], xi.shape[0]
    rho_o, rho_i = 1.0, 2.0
    m_o = rho_o * 0.25 / n_o   # outer volume 1 x 0.5 x 0.5
    m_i = rho_i * 0.25 / n_i   # inner volume 1 x 0.5 x 0.5
    x = np.concatenate([xo, xi])
    y = np.concatenate([yo, yi])
    z = np.concatenate([zo, zi])
    inner = np.concatenate([np.zeros(n_o, bool), np.ones(n_i, bool)])
    vx = np.where(inner, 0.5, -0.5)
    vy = 0.01 * np.sin(4.0 * np.pi * x)
    vz = np.zeros(x.shape[0])
    h = np.where(inner, h_for_neighbors(di, ng), h_for_neighbors(do, ng))
    m = np.where(inner, m_i, m_o)
    u = np.where(inner, pressure / ((gamma - 1.0) * rho_i), pressure / ((gamma - 1.0) * rho_o))
    return _finish(x, y, z, vx, vy, vz, h, m, u, (0.0, 0.0, 0.0), (1.0, 1.0, 0.5), (1, 1, 1),
                   rng=rng, shuffle=shuffle)


def ensemble_sides(n_boxes: int = 256, lo: int = 8, hi: int = 48, seed_index: int = 4):
    """Per-box lattice sides drawn log-uniformly in [lo, hi] and per-box alpha
    uniform in [0.5, 1.5]."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    sides = np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), n_boxes))).astype(int)
    alphas = rng.uniform(0.5, 1.5, n_boxes)
    return sides, alphas


def ensemble(n_boxes: int = 256, lo: int = 8, hi: int = 48, seed_index: int = 4):
    """List of (state, alpha) for the batched-ensemble workload; box k uses
    the jittered-box recipe with seed index 1000 + k."""
    sides, alphas = ensemble_sides(n_boxes, lo, hi, seed_index)
    return [(jittered_box(int(s), seed_index=1000 + k), float(a))
            for k, (s, a) in enumerate(zip(sides, alphas))]


def to_numpy_state(s: dict) -> dict:
    return {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in s.items()}


def uniform_sphere(side: int = 124, seed_index: int = 5, jitter: float = 0.1, ng: int = NG_TARGET,
                   shuffle=True):
    """Uniform sphere of radius 1 and mass 1 from a jittered cubic lattice of
    spacing 2/side (side = 124 gives about 10^6 particles), at rest, u = 1,
    all axes open."""
    rng = np.random.default_rng(SEED_BASE + seed_index)
    dx = 2.0 / side
    X, Y, Z = _lattice(side, side, side, (-1.0, -1.0, -1.0), dx)
    X = X + rng.uniform(-jitter, jitter, X.shape) * dx
    Y = Y + rng.uniform(-jitter, jitter, Y.shape) * dx
    Z = Z + rng.uniform(-jitter, jitter, Z.shape) * dx
    inside = X * X + Y * Y + Z * Z < 1.0
    X, Y, Z = X[inside], Y[inside], Z[inside]
    n = X.shape[0]
    zeros = np.zeros(n)
    return _finish(X, Y, Z, zeros, zeros.copy(), zeros.copy(), np.full(n, h_for_neighbors(dx, ng)),
                   np.full(n, 1.0 / n), np.ones(n), (-1.0, -1.0, -1.0), (1.0, 1.0, 1.0), (0, 0, 0),
                   rng=rng, shuffle=shuffle)
