"""Plain FP64 CPU oracle of the SPH per-step pipeline (test infrastructure).

The arithmetic lives in ``sph_oracle.c`` (plain C, no fused multiply-add,
libm ``sin``/``sqrt``/``cbrt``), written from the paper's section 4.1 equations
and the readings stated there.  This module only compiles it and marshals
numpy arrays.  It is the correctness reference for the CUDA library and is used
by the tests, the smoke check and the benchmark's CPU-baseline leg only; the
product path never imports it, and it imports nothing from the product.

Arrays are FP64 structure-of-arrays indexed by particle index.  Neighbour lists
are int64 particle indices, sorted ascending, self excluded.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import sys
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

OK, INVALID_ARG, NB_OVERFLOW, SINGULAR_IAD, NONFINITE = 0, -1, -3, -4, -5


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` with gcc (OpenMP, -ffp-contract=off)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC", "-shared",
           "-std=c11", "-o", _LIB + ".tmp", _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


class _Box(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("periodic", C.c_int * 3)]


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        d, i64, i32, cint = C.c_double, C.c_int64, C.c_int32, C.c_int
        P = C.c_void_p
        lib.oracle_kernel_norm.restype = d
        lib.oracle_kernel_norm.argtypes = [d]
        lib.oracle_kernel_W.restype = d
        lib.oracle_kernel_W.argtypes = [d, d, d, d]
        lib.oracle_kernel_dWdv.restype = d
        lib.oracle_kernel_dWdv.argtypes = [d, d, d, d]
        lib.oracle_kernel_dWdh.restype = d
        lib.oracle_kernel_dWdh.argtypes = [d, d, d, d]
        lib.oracle_set_kernel_mode.restype = None
        lib.oracle_set_kernel_mode.argtypes = [cint, d]
        lib.oracle_kernel_W_table.restype = d
        lib.oracle_kernel_W_table.argtypes = [d, d, d, d]
        lib.oracle_find_neighbors.restype = cint
        lib.oracle_find_neighbors.argtypes = [C.POINTER(_Box), i64, P, P, P, P, i64, P, cint, cint, P, P]
        lib.oracle_density_eos.restype = None
        lib.oracle_density_eos.argtypes = [C.POINTER(_Box), P, P, P, P, P, P, i64, P, P, P, cint,
                                           d, d, d, P, P, P, P]
        lib.oracle_iad.restype = cint
        lib.oracle_iad.argtypes = [C.POINTER(_Box), P, P, P, P, P, P, i64, P, P, P, cint, d, d, P, P]
        lib.oracle_momentum_energy.restype = None
        lib.oracle_momentum_energy.argtypes = [C.POINTER(_Box), P, P, P, P, P, P, P, P, P, P, P, P,
                                               P, i64, P, P, P, cint, d, d, d, P, P, P, P, P, P,
                                               P, P]
        lib.oracle_timestep.restype = d
        lib.oracle_timestep.argtypes = [i64, P, P, d, d, d]
        lib.oracle_timestep_u.restype = d
        lib.oracle_timestep_u.argtypes = [i64, P, P, P, P, d, d, d, d]
        lib.oracle_update.restype = None
        lib.oracle_update.argtypes = [C.POINTER(_Box), i64] + [P] * 17 + [d, d, cint]
        lib.oracle_diagnostics.restype = None
        lib.oracle_diagnostics.argtypes = [i64] + [P] * 9
        lib.oracle_any_nonfinite.restype = cint
        lib.oracle_gravity_direct.restype = None
        lib.oracle_gravity_direct.argtypes = [i64, P, P, P, P, d, d, i64, P, P, P, P]
        lib.oracle_gravity_tree.restype = cint
        lib.oracle_gravity_tree.argtypes = [i64, P, P, P, P, P, d, d, d, i64, P, P, P, P, P]
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = cint
        lib.oracle_set_num_threads.argtypes = [cint]
        lib.oracle_set_num_threads.restype = cint
        lib.oracle_any_nonfinite.argtypes = [i64, P]
        _lib = lib
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class Box:
    """Simulation box: corners and per-axis periodicity (open axes ignore lo/hi)."""
    lo: tuple = (0.0, 0.0, 0.0)
    hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (1, 1, 1)

    def c(self):
        b = _Box()
        for k in range(3):
            b.lo[k], b.hi[k], b.periodic[k] = float(self.lo[k]), float(self.hi[k]), int(self.periodic[k])
        return b


@dataclass
class Params:
    """Physical and numerical parameters of a step (the paper's section 4.1
    quantities plus the readings for the unprinted choices)."""
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    courant: float = 0.2
    dt_growth: float = 1.1
    sinc_n: float = 6.0
    ng_target: int = 100
    max_nb: int = 160
    gradh: int = 0          # 1: grad-h terms Omega in Eqs. 2-3
    kernel_mode: int = 0    # 0: exact sinc kernel; 1: 20,000-entry table (section 4.5)
    energy_dt: float = 0.0  # > 0: dt <= energy_dt * min u / |du| (opt-in reading)


def num_threads() -> int:
    """Threads the oracle's per-particle loops run on."""
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> int:
    """Sets the threads of the per-particle loops; returns the count in effect."""
    return int(_load().oracle_set_num_threads(int(n)))


def kernel_norm(sinc_n: float = 6.0) -> float:
    """B_n such that the sinc kernel of Eq. 6 integrates to one in 3-D."""
    return _load().oracle_kernel_norm(float(sinc_n))


def kernel_W(v: float, h: float, sinc_n: float = 6.0, Bn: float | None = None) -> float:
    """W(v, h) of Eq. 6 (d = 3)."""
    if Bn is None:
        Bn = kernel_norm(sinc_n)
    return _load().oracle_kernel_W(float(v), float(h), float(sinc_n), float(Bn))


def kernel_W_table(v: float, h: float, sinc_n: float = 6.0, Bn: float | None = None) -> float:
    """W(v, h) from the 20,000-entry table with linear interpolation."""
    if Bn is None:
        Bn = kernel_norm(sinc_n)
    return _load().oracle_kernel_W_table(float(v), float(h), float(sinc_n), float(Bn))


def _mode(params):
    """Select the oracle's kernel evaluation for the next call."""
    _load().oracle_set_kernel_mode(int(getattr(params, "kernel_mode", 0)), float(params.sinc_n))


def kernel_dWdv(v: float, h: float, sinc_n: float = 6.0, Bn: float | None = None) -> float:
    """dW/dv of Eq. 6 at fixed h."""
    if Bn is None:
        Bn = kernel_norm(sinc_n)
    return _load().oracle_kernel_dWdv(float(v), float(h), float(sinc_n), float(Bn))


def kernel_dWdh(v: float, h: float, sinc_n: float = 6.0, Bn: float | None = None) -> float:
    """dW/dh of Eq. 6 at fixed separation (v = r / h)."""
    if Bn is None:
        Bn = kernel_norm(sinc_n)
    return _load().oracle_kernel_dWdh(float(v), float(h), float(sinc_n), float(Bn))


def find_neighbors(box: Box, x, y, z, h, targets=None, brute=False, max_nb=160):
    """Neighbour lists (b != a, r_ab^2 < (2 h_a)^2).  Returns (rc, nn, nbr)."""
    x, y, z, h = map(_f64, (x, y, z, h))
    n = x.shape[0]
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = n if t is None else t.shape[0]
    nn = np.zeros(nt, dtype=np.int32)
    nbr = np.full((nt, max_nb), -1, dtype=np.int64)
    b = box.c()
    rc = _load().oracle_find_neighbors(C.byref(b), n, _p(x), _p(y), _p(z), _p(h), nt, _p(t),
                                       1 if brute else 0, max_nb, _p(nn), _p(nbr))
    return rc, nn, nbr


def density_eos(box: Box, s: dict, nn, nbr, params: Params, targets=None, Bn=None,
                with_omega=False):
    """Eq. 1 density (self term included) and the ideal-gas EOS.  Returns
    (rho, p, c), plus the grad-h terms Omega when with_omega."""
    if Bn is None:
        Bn = kernel_norm(params.sinc_n)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = s["x"].shape[0] if t is None else t.shape[0]
    rho, p, c = (np.empty(nt) for _ in range(3))
    omega = np.empty(nt) if with_omega else None
    b = box.c()
    _mode(params)
    _load().oracle_density_eos(C.byref(b), _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(s["h"]),
                               _p(s["m"]), _p(s["u"]), nt, _p(t), _p(nn), _p(nbr), nbr.shape[1],
                               params.sinc_n, Bn, params.gamma, _p(rho), _p(p), _p(c), _p(omega))
    return (rho, p, c, omega) if with_omega else (rho, p, c)


def iad(box: Box, s: dict, rho_full, nn, nbr, params: Params, targets=None, Bn=None):
    """IAD matrix C = tau^{-1} (6 unique entries) and tau.  Returns (rc, C6, tau6)."""
    if Bn is None:
        Bn = kernel_norm(params.sinc_n)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = s["x"].shape[0] if t is None else t.shape[0]
    C6 = np.empty((nt, 6))
    T6 = np.empty((nt, 6))
    rho_full = _f64(rho_full)
    b = box.c()
    _mode(params)
    rc = _load().oracle_iad(C.byref(b), _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(s["h"]), _p(s["m"]),
                            _p(rho_full), nt, _p(t), _p(nn), _p(nbr), nbr.shape[1], params.sinc_n, Bn,
                            _p(C6), _p(T6))
    return rc, C6, T6


def momentum_energy(box: Box, s: dict, rho_full, p_full, c_full, iad_full, nn, nbr, params: Params,
                    targets=None, Bn=None, av_force=None, record_av=False, omega_full=None):
    """Eqs. 2-5.  Returns dict with ax, ay, az, du and the scales sa, sdu.
    ``av_force`` (int8, shape of ``nbr``) imposes the viscosity switch of Eq. 5
    per list entry; ``record_av`` returns the switch as decided in ``av``;
    ``omega_full`` holds the grad-h terms (None: Omega = 1)."""
    if Bn is None:
        Bn = kernel_norm(params.sinc_n)
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = s["x"].shape[0] if t is None else t.shape[0]
    out = {k: np.empty(nt) for k in ("ax", "ay", "az", "du", "sa", "sdu")}
    rho_full, p_full, c_full = map(_f64, (rho_full, p_full, c_full))
    iad_full = np.ascontiguousarray(iad_full, dtype=np.float64).reshape(-1, 6)
    omega_full = None if omega_full is None else _f64(omega_full)
    if av_force is not None:
        av_force = np.ascontiguousarray(av_force, dtype=np.int8)
        assert av_force.shape == nbr.shape
    av = np.zeros(nbr.shape, dtype=np.int8) if record_av else None
    b = box.c()
    _mode(params)
    _load().oracle_momentum_energy(
        C.byref(b), _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(s["vx"]), _p(s["vy"]), _p(s["vz"]),
        _p(s["h"]), _p(s["m"]), _p(rho_full), _p(p_full), _p(c_full), _p(iad_full),
        _p(omega_full), nt, _p(t),
        _p(nn), _p(nbr), nbr.shape[1], params.sinc_n, Bn, params.alpha, _p(av_force), _p(av),
        _p(out["ax"]), _p(out["ay"]), _p(out["az"]), _p(out["du"]), _p(out["sa"]), _p(out["sdu"]))
    if record_av:
        out["av"] = av
    return out


def timestep(h, c, params: Params, dt_prev: float, u=None, du=None) -> float:
    """Courant time step with growth cap; with params.energy_dt > 0 also the
    energy-rate limit energy_dt * min u / |du| (u, du required then)."""
    h, c = _f64(h), _f64(c)
    if params.energy_dt > 0.0:
        u, du = _f64(u), _f64(du)
        return _load().oracle_timestep_u(h.shape[0], _p(h), _p(c), _p(u), _p(du), params.courant,
                                         float(params.energy_dt), params.dt_growth, float(dt_prev))
    return _load().oracle_timestep(h.shape[0], _p(h), _p(c), params.courant, params.dt_growth,
                                   float(dt_prev))


def update(box: Box, s: dict, ax, ay, az, du, nn, dt: float, dt_prev: float, ng_target: int):
    """Integrator and smoothing-length update, in place on the state dict."""
    ax, ay, az, du = map(_f64, (ax, ay, az, du))
    nn = np.ascontiguousarray(nn, dtype=np.int32)
    b = box.c()
    _load().oracle_update(C.byref(b), s["x"].shape[0], _p(s["x"]), _p(s["y"]), _p(s["z"]),
                          _p(s["vx"]), _p(s["vy"]), _p(s["vz"]), _p(s["vxh"]), _p(s["vyh"]),
                          _p(s["vzh"]), _p(s["u"]), _p(s["du_prev"]), _p(s["h"]), _p(ax), _p(ay),
                          _p(az), _p(du), _p(nn), float(dt), float(dt_prev), int(ng_target))


def diagnostics(s: dict) -> np.ndarray:
    """{Px, Py, Pz, E_kin, E_int, Lx, Ly, Lz} by compensated FP64 sums."""
    out = np.zeros(8)
    _load().oracle_diagnostics(s["x"].shape[0], _p(s["x"]), _p(s["y"]), _p(s["z"]), _p(s["vx"]),
                               _p(s["vy"]), _p(s["vz"]), _p(s["m"]), _p(s["u"]), _p(out))
    return out


STATE_KEYS = ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u", "du_prev")


def copy_state(s: dict) -> dict:
    return {k: (np.array(v, copy=True) if isinstance(v, np.ndarray) else v) for k, v in s.items()}


def outputs(box: Box, s: dict, params: Params, brute=False, record_av=False):
    """Every per-particle output of one step on the given state (no update):
    neighbour lists, rho, P, c, C (IAD), a, du and the normalisation scales.
    Returns (rc, dict)."""
    rc, nn, nbr = find_neighbors(box, s["x"], s["y"], s["z"], s["h"], brute=brute,
                                 max_nb=params.max_nb)
    if rc != OK:
        return rc, {"nn": nn, "nbr": nbr}
    Bn = kernel_norm(params.sinc_n)
    omega = None
    if params.gradh:
        rho, p, c, omega = density_eos(box, s, nn, nbr, params, Bn=Bn, with_omega=True)
    else:
        rho, p, c = density_eos(box, s, nn, nbr, params, Bn=Bn)
    rc_iad, C6, T6 = iad(box, s, rho, nn, nbr, params, Bn=Bn)
    me = momentum_energy(box, s, rho, p, c, C6, nn, nbr, params, Bn=Bn, record_av=record_av,
                         omega_full=omega)
    out = {"nn": nn, "nbr": nbr, "rho": rho, "p": p, "c": c, "iad": C6, "tau": T6}
    if omega is not None:
        out["omega"] = omega
    out.update(me)
    return rc_iad, out


def step(box: Box, s: dict, params: Params, dt_prev: float, brute=False, record_av=False):
    """One full step in place on ``s`` (find neighbours, density + EOS, IAD,
    momentum/energy, time step, update, smoothing length).  Returns
    (rc, dt, outputs-of-the-step)."""
    rc, out = outputs(box, s, params, brute=brute, record_av=record_av)
    if rc not in (OK,):
        return rc, float("nan"), out
    dt = timestep(s["h"], out["c"], params, dt_prev, u=s["u"], du=out["du"])
    update(box, s, out["ax"], out["ay"], out["az"], out["du"], out["nn"], dt, dt_prev,
           params.ng_target)
    return OK, dt, out


def sampled_outputs(box: Box, s: dict, params: Params, sample):
    """Outputs of one step for a sample of target particles only, on a state of
    any size: density on the 2-ring of the sample, IAD on its 1-ring, momentum
    on the sample.  Returns (rc, dict of per-sample arrays)."""
    sample = np.ascontiguousarray(sample, dtype=np.int64)
    n = s["x"].shape[0]
    Bn = kernel_norm(params.sinc_n)
    rc, nn0, nbr0 = find_neighbors(box, s["x"], s["y"], s["z"], s["h"], targets=sample,
                                   max_nb=params.max_nb)
    if rc != OK:
        return rc, None
    ring1 = np.unique(np.concatenate([sample, nbr0[nbr0 >= 0]]))
    rc, nn1, nbr1 = find_neighbors(box, s["x"], s["y"], s["z"], s["h"], targets=ring1,
                                   max_nb=params.max_nb)
    if rc != OK:
        return rc, None
    ring2 = np.unique(np.concatenate([ring1, nbr1[nbr1 >= 0]]))
    rc, nn2, nbr2 = find_neighbors(box, s["x"], s["y"], s["z"], s["h"], targets=ring2,
                                   max_nb=params.max_nb)
    if rc != OK:
        return rc, None
    rho = np.full(n, np.nan)
    pp = np.full(n, np.nan)
    cc = np.full(n, np.nan)
    om = np.full(n, np.nan) if params.gradh else None
    dens = density_eos(box, s, nn2, nbr2, params, targets=ring2, Bn=Bn, with_omega=bool(params.gradh))
    rho[ring2], pp[ring2], cc[ring2] = dens[:3]
    if params.gradh:
        om[ring2] = dens[3]
    iadf = np.full((n, 6), np.nan)
    rc_iad, C1, _ = iad(box, s, rho, nn1, nbr1, params, targets=ring1, Bn=Bn)
    iadf[ring1] = C1
    me = momentum_energy(box, s, rho, pp, cc, iadf, nn0, nbr0, params, targets=sample, Bn=Bn,
                         omega_full=om)
    out = {"nn": nn0, "nbr": nbr0, "rho": rho[sample], "p": pp[sample], "c": cc[sample],
           "iad": iadf[sample]}
    if params.gradh:
        out["omega"] = om[sample]
    out.update(me)
    return rc_iad, out


def gravity_direct(s: dict, G: float = 1.0, eps: float = 0.0, targets=None):
    """Softened Newtonian self-gravity by direct summation (the definition).
    Returns g (nt, 3)."""
    x, y, z, m = (_f64(s[k]) for k in ("x", "y", "z", "m"))
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = x.shape[0] if t is None else t.shape[0]
    g = np.empty((3, nt))
    _load().oracle_gravity_direct(x.shape[0], _p(x), _p(y), _p(z), _p(m), float(G), float(eps),
                                  nt, _p(t), _p(g[0]), _p(g[1]), _p(g[2]))
    return g.T.copy()


def gravity_tree(s: dict, G: float = 1.0, eps: float = 0.0, theta: float = 0.5, targets=None):
    """Self-gravity by the multipole tree on the neighbour grid's cells.
    Returns (rc, g (nt, 3), [node interactions, particle interactions])."""
    x, y, z, h, m = (_f64(s[k]) for k in ("x", "y", "z", "h", "m"))
    t = None if targets is None else np.ascontiguousarray(targets, dtype=np.int64)
    nt = x.shape[0] if t is None else t.shape[0]
    g = np.empty((3, nt))
    stats = np.zeros(2, dtype=np.int64)
    rc = _load().oracle_gravity_tree(x.shape[0], _p(x), _p(y), _p(z), _p(h), _p(m), float(G),
                                     float(eps), float(theta), nt, _p(t), _p(g[0]), _p(g[1]),
                                     _p(g[2]), _p(stats))
    return rc, g.T.copy(), stats
