"""Differentiable SPH rollout on one GPU (libsph's sph_adjoint_* entry
points): K FP64 steps plus a final density pass, with hand-written adjoint
kernels for the reverse pass and a state checkpoint every few steps.

``Rollout`` owns the library context; ``rollout(...)`` is the
``torch.autograd.Function`` front end: it returns the final positions,
velocities, internal energies and densities as tensors whose gradients flow
back to the initial positions, velocities, internal energies and the
viscosity alpha of Eq. 5.  Neighbour lists, smoothing lengths, time steps and
the viscosity switch are held at their forward values (the derivative of the
rollout wherever none of them changes).  PyTorch provides device memory and
the stream only; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from ._lib import SphState
from .sim import Params, _stream_ptr

FINAL = ("x", "y", "z", "vx", "vy", "vz", "u", "rho")
GRAD_INIT = ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "u", "du_prev")


class Rollout:
    """A rollout of ``steps`` FP64 steps for up to ``n_max`` particles, with a
    checkpoint every ``checkpoint_every`` steps."""

    def __init__(self, n_max: int, steps: int, checkpoint_every: int = 5,
                 params: Params | None = None, device: str = "cuda:0"):
        self.lib = _lib.load()
        self.device = torch.device(device)
        params = params or Params()
        params.precision = "fp64"
        self.params = params
        self.n_max, self.steps, self.every = int(n_max), int(steps), int(checkpoint_every)
        self._cp = params.c()
        self.ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.sph_adjoint_init(C.byref(self._cp), self.n_max, self.steps, self.every,
                                           C.byref(self.ctx))
        if rc != _lib.SPH_OK:
            raise _lib.SphError(rc, "sph_adjoint_init")
        self._n = 0
        self.forwards = 0       # forward rollouts run so far (the tape holds the last one)

    def _err(self, rc):
        if rc != _lib.SPH_OK:
            raise _lib.SphError(rc, (self.lib.sph_adjoint_last_error(self.ctx) or b"").decode())

    def forward(self, state: dict, alpha: float, dt_prev0: float = 0.0) -> torch.Tensor:
        """state: dict of contiguous FP64 device tensors (n,) for the 13 state
        fields.  Returns final (8, n): x, y, z, vx, vy, vz, u, rho."""
        n = int(state["x"].shape[0])
        st = SphState()
        keep = {}
        for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u", "du_prev"):
            t = state[k]
            assert t.dtype == torch.float64 and t.device == self.device and t.numel() == n
            t = t.contiguous()
            keep[k] = t
            setattr(st, k, t.data_ptr())
        st.n = n
        out = torch.empty(8, n, dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_adjoint_forward(self.ctx, C.byref(st), float(dt_prev0),
                                                   float(alpha), C.c_void_p(out.data_ptr()),
                                                   _stream_ptr()))
        self._n = n
        self.forwards += 1
        return out

    def backward(self, g_final: torch.Tensor):
        """g_final (8, n) = dL/d(final).  Returns (g_init (11, n), g_alpha (0-d))."""
        g = g_final.to(device=self.device, dtype=torch.float64).contiguous()
        n = self._n or g.shape[-1]              # before a forward the library reports ORDER
        assert g.shape == (8, n)
        gi = torch.empty(11, n, dtype=torch.float64, device=self.device)
        ga = torch.empty((), dtype=torch.float64, device=self.device)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_adjoint_backward(self.ctx, C.c_void_p(g.data_ptr()),
                                                    C.c_void_p(gi.data_ptr()),
                                                    C.c_void_p(ga.data_ptr()), _stream_ptr()))
        return gi, ga

    def time_steps(self) -> np.ndarray:
        dt = np.zeros(self.steps)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_adjoint_time_steps(self.ctx, dt.ctypes.data_as(C.c_void_p)))
        return dt

    def info(self) -> dict:
        out = np.zeros(4, dtype=np.int64)
        self._err(self.lib.sph_adjoint_info(self.ctx, out.ctypes.data_as(C.c_void_p)))
        return {"bytes": int(out[0]), "launches": int(out[1]), "recomputed_steps": int(out[2]),
                "backward_passes": int(out[3])}

    def close(self):
        if getattr(self, "ctx", None):
            with torch.cuda.device(self.device):
                self.lib.sph_adjoint_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SphRolloutFn(torch.autograd.Function):
    """(x0 (n,3), v0 (n,3), u0 (n), alpha (0-d)) -> (x (n,3), v (n,3), u (n),
    rho (n)) after the rollout.  v0 seeds both the velocity and the half-step
    velocity of the integrator, so its gradient is the sum of the two."""

    @staticmethod
    def forward(ctx, x0, v0, u0, alpha, ro: Rollout, h, m, du_prev, dt_prev0):
        state = {"x": x0[:, 0], "y": x0[:, 1], "z": x0[:, 2],
                 "vx": v0[:, 0], "vy": v0[:, 1], "vz": v0[:, 2],
                 "vxh": v0[:, 0], "vyh": v0[:, 1], "vzh": v0[:, 2],
                 "h": h, "m": m, "u": u0, "du_prev": du_prev}
        state = {k: v.detach().contiguous() for k, v in state.items()}
        fin = ro.forward(state, float(alpha), float(dt_prev0))
        ctx.ro = ro
        ctx.forward_id = ro.forwards
        x = fin[0:3].t().contiguous()
        v = fin[3:6].t().contiguous()
        return x, v, fin[6].clone(), fin[7].clone()

    @staticmethod
    def backward(ctx, gx, gv, gu, grho):
        ro = ctx.ro
        if ro.forwards != ctx.forward_id:
            # the Rollout's tape holds a newer forward than this graph's
            raise RuntimeError("this Rollout ran another forward since the one being "
                               "differentiated; a Rollout holds the tape of its last forward "
                               "only (use one Rollout per pending backward)")
        n = ro._n
        dev = ro.device

        def z(t, shape):
            return torch.zeros(shape, dtype=torch.float64, device=dev) if t is None else t

        g = torch.cat([z(gx, (n, 3)).t(), z(gv, (n, 3)).t(), z(gu, (n,))[None],
                       z(grho, (n,))[None]], 0)
        gi, ga = ro.backward(g)
        gx0 = gi[0:3].t().contiguous()
        gv0 = (gi[3:6] + gi[6:9]).t().contiguous()
        return gx0, gv0, gi[9].clone(), ga, None, None, None, None, None


def rollout(x0, v0, u0, alpha, ro: Rollout, h, m, du_prev=None, dt_prev0: float = 0.0):
    """Differentiable K-step rollout (see SphRolloutFn)."""
    if du_prev is None:
        du_prev = torch.zeros_like(u0)
    if not torch.is_tensor(alpha):
        alpha = torch.tensor(float(alpha), dtype=torch.float64, device=x0.device)
    return SphRolloutFn.apply(x0, v0, u0, alpha, ro, h, m, du_prev, dt_prev0)
