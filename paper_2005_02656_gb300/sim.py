"""Python front end of libsph: device state in torch tensors, calls through the
C ABI.  PyTorch only provides device memory and the current CUDA stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib
from ._lib import SphParams, SphState, check

PERSISTENT = ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u", "du_prev")
OUTPUTS = ("rho", "p", "c", "ax", "ay", "az", "du")


@dataclass
class Params:
    """Mirror of sph_params (include/sph.h)."""
    box_lo: tuple = (0.0, 0.0, 0.0)
    box_hi: tuple = (1.0, 1.0, 1.0)
    periodic: tuple = (1, 1, 1)
    gamma: float = 5.0 / 3.0
    alpha: float = 1.0
    courant: float = 0.2
    dt_growth: float = 1.1
    ng_target: int = 100
    max_nb: int = 160
    sinc_n: float = 6.0
    precision: str = "fp64"   # "fp64" | "fp32_mixed"
    gradh: int = 0            # 1: grad-h terms Omega in Eqs. 2-3
    kernel_mode: str = "exact"  # "exact" | "table" (section 4.5: 20,000-entry table)
    pair_mode: str = "staged"   # FP32-mixed pair sums: "staged" (cell-staged candidates
                                # and hit masks) | "lists" (int32 neighbour lists)
    energy_dt: float = 0.0      # > 0: dt <= energy_dt * min u / |du| (opt-in energy-rate limit)
    angular_sums: int = 0       # 1: each step also sums the angular momentum (last_diagnostics()[5:8])

    def c(self) -> SphParams:
        p = SphParams()
        for k in range(3):
            p.box_lo[k] = float(self.box_lo[k])
            p.box_hi[k] = float(self.box_hi[k])
            p.periodic[k] = int(self.periodic[k])
        p.gamma, p.alpha, p.courant, p.dt_growth = self.gamma, self.alpha, self.courant, self.dt_growth
        p.ng_target, p.max_nb, p.sinc_n = int(self.ng_target), int(self.max_nb), float(self.sinc_n)
        p.precision = {"fp64": _lib.SPH_FP64, "fp32_mixed": _lib.SPH_FP32_MIXED}[self.precision]
        p.kernel_mode = {"exact": _lib.SPH_KERNEL_EXACT, "table": _lib.SPH_KERNEL_TABLE}[self.kernel_mode]
        p.gradh = int(self.gradh)
        p.pair_mode = {"staged": _lib.SPH_PAIRS_STAGED, "lists": _lib.SPH_PAIRS_LISTS}[self.pair_mode]
        p.energy_dt = float(self.energy_dt)
        p.angular_sums = int(self.angular_sums)
        return p


def _stream_ptr():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def measure_fp32_peak() -> float:
    """FP32 fused-multiply-add rate of the current device in TFLOP/s, measured
    by the library's probe kernel on the current stream (sph_measure_fp32_peak)."""
    lib = _lib.load()
    out = C.c_double(0.0)
    check(lib, None, lib.sph_measure_fp32_peak(C.byref(out), _stream_ptr()))
    return float(out.value)


class SphSim:
    """A particle state on one GPU and a libsph context.

    ``state`` is a dict of numpy arrays as produced by ``sph_inputs`` (keys
    x y z vx vy vz vxh vyh vzh h m u du_prev id, plus lo/hi/periodic).
    """

    def __init__(self, state: dict, params: Params | None = None, n_max: int | None = None,
                 device: str = "cuda:0", **overrides):
        self.lib = _lib.load()
        self.device = torch.device(device)
        if params is None:
            params = Params(box_lo=state["lo"], box_hi=state["hi"], periodic=state["periodic"])
        for k, v in overrides.items():
            setattr(params, k, v)
        self.params = params
        n = int(state["x"].shape[0])
        self.n = n
        self.n_max = int(n_max or n)
        with torch.cuda.device(self.device):
            self.ctx = C.c_void_p()
            self._cp = params.c()
            check(self.lib, None, self.lib.sph_init(C.byref(self._cp), self.n_max, C.byref(self.ctx)))
            dev = self.device
            self.t = {}
            for k in PERSISTENT:
                self.t[k] = torch.as_tensor(np.ascontiguousarray(state[k], dtype=np.float64)).to(dev)
            self.t["id"] = torch.as_tensor(np.ascontiguousarray(state["id"], dtype=np.int64)).to(dev)
            for k in OUTPUTS:
                self.t[k] = torch.zeros(n, dtype=torch.float64, device=dev)
            self.t["iad"] = torch.zeros(6 * n, dtype=torch.float64, device=dev)
            self.t["omega"] = torch.ones(n, dtype=torch.float64, device=dev)  # grad-h terms
            self.dt = torch.zeros(1, dtype=torch.float64, device=dev)
        self._st = SphState()
        self._bind()

    # -- marshalling --
    def _bind(self):
        for k in _lib.STATE_FIELDS:
            setattr(self._st, k, self.t[k].data_ptr())
        self._st.id = self.t["id"].data_ptr()
        self._st.n = self.n

    def _call(self, fn, *args):
        with torch.cuda.device(self.device):
            rc = fn(self.ctx, *args)
        return check(self.lib, self.ctx, rc)

    def close(self):
        if getattr(self, "ctx", None):
            with torch.cuda.device(self.device):
                torch.cuda.synchronize()
                self.lib.sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- stages --
    def set_params(self, **kw):
        for k, v in kw.items():
            setattr(self.params, k, v)
        self._cp = self.params.c()
        self._call(self.lib.sph_set_params, C.byref(self._cp))

    def find_neighbors(self):
        self._call(self.lib.sph_find_neighbors, C.byref(self._st), _stream_ptr())

    def density(self):
        self._call(self.lib.sph_density, C.byref(self._st), _stream_ptr())

    def iad(self):
        self._call(self.lib.sph_iad, C.byref(self._st), _stream_ptr())

    def momentum_energy(self):
        self._call(self.lib.sph_momentum_energy, C.byref(self._st), _stream_ptr())

    def step(self, steps: int = 1):
        for _ in range(steps):
            self._call(self.lib.sph_step, C.byref(self._st), C.c_void_p(self.dt.data_ptr()),
                       _stream_ptr())

    def gravity(self, G: float = 1.0, eps: float = 0.0, theta: float = 0.5):
        """Self-gravity by the multipole tree (sph_gravity), in the sim's
        precision; sorts the state.  Returns (g (n, 3) FP64 device tensor in
        the current order, [node, particle] interactions)."""
        g = torch.empty(3, self.n, dtype=torch.float64, device=self.device)
        cnt = np.zeros(2, dtype=np.int64)
        self._call(self.lib.sph_gravity, C.byref(self._st), float(G), float(eps), float(theta),
                   C.c_void_p(g[0].data_ptr()), C.c_void_p(g[1].data_ptr()),
                   C.c_void_p(g[2].data_ptr()), cnt.ctypes.data_as(C.c_void_p), _stream_ptr())
        return g.t(), cnt

    def get_neighbors(self):
        """(counts[n] int32, ids[n, max_nb] int64) in id space, rows by current position."""
        mb = self.params.max_nb
        counts = torch.zeros(self.n, dtype=torch.int32, device=self.device)
        ids = torch.full((self.n, mb), -1, dtype=torch.int64, device=self.device)
        self._call(self.lib.sph_get_neighbors, C.byref(self._st), C.c_void_p(counts.data_ptr()),
                   C.c_void_p(ids.data_ptr()), _stream_ptr())
        return counts, ids

    def diagnostics(self) -> np.ndarray:
        out = np.zeros(8)
        self._call(self.lib.sph_diagnostics, C.byref(self._st), out.ctypes.data_as(C.c_void_p),
                   _stream_ptr())
        return out

    def last_diagnostics(self) -> np.ndarray:
        out = np.zeros(12)
        self._call(self.lib.sph_last_diagnostics, out.ctypes.data_as(C.c_void_p), _stream_ptr())
        return out

    def error_word(self) -> int:
        f = C.c_uint32(0)
        self._call(self.lib.sph_error_word, C.byref(f))
        return int(f.value)

    def kernel_norm(self) -> float:
        return float(self.lib.sph_kernel_norm(self.ctx))

    def launch_count(self) -> int:
        return int(self.lib.sph_launch_count(self.ctx))

    def stats(self) -> dict:
        out = np.zeros(6, dtype=np.uint64)
        self._call(self.lib.sph_stats, out.ctypes.data_as(C.c_void_p))
        return {"candidates": int(out[0]), "exact_tests": int(out[1]), "pairs": int(out[2]),
                "particle_updates": int(out[3]), "staged_slots": int(out[4]),
                "mask_words": int(out[5])}

    def profile(self, enable: bool = True):
        self._call(self.lib.sph_profile, 1 if enable else 0)

    def stage_times(self):
        """(dict stage -> accumulated ms, number of steps) since the last call."""
        ms = np.zeros(len(_lib.STAGES))
        steps = np.zeros(1, dtype=np.int64)
        self._call(self.lib.sph_stage_times, ms.ctypes.data_as(C.c_void_p),
                   steps.ctypes.data_as(C.c_void_p))
        return dict(zip(_lib.STAGES, ms.tolist())), int(steps[0])

    # -- host views --
    def to_numpy(self, by_id: bool = True) -> dict:
        """State and outputs as numpy arrays, ordered by particle id if by_id."""
        torch.cuda.synchronize(self.device)
        out = {k: self.t[k].cpu().numpy() for k in PERSISTENT + OUTPUTS + ("id", "omega")}
        out["iad"] = self.t["iad"].cpu().numpy().reshape(-1, 6)
        if by_id:
            order = np.argsort(out["id"], kind="stable")
            out = {k: v[order] for k, v in out.items()}
        return out

    def set_state(self, state: dict):
        """Overwrite the persistent state (same n) from numpy arrays."""
        for k in PERSISTENT:
            self.t[k].copy_(torch.as_tensor(np.ascontiguousarray(state[k], dtype=np.float64)))
        self.t["id"].copy_(torch.as_tensor(np.ascontiguousarray(state["id"], dtype=np.int64)))
        self.dt.zero_()


class HostStepper:
    """sph_step_host on pinned host arrays (the end-to-end path for callers
    whose state lives in host memory)."""

    def __init__(self, state: dict, params: Params | None = None, n_max: int | None = None,
                 device: str = "cuda:0", outputs: bool = False, pinned: bool = True):
        self.lib = _lib.load()
        self.device = torch.device(device)
        if params is None:
            params = Params(box_lo=state["lo"], box_hi=state["hi"], periodic=state["periodic"])
        self.params = params
        self.n = int(state["x"].shape[0])
        with torch.cuda.device(self.device):
            self.ctx = C.c_void_p()
            self._cp = params.c()
            check(self.lib, None, self.lib.sph_init(C.byref(self._cp), int(n_max or self.n),
                                                    C.byref(self.ctx)))
        # pinned arrays let the library overlap its copies and write the new
        # state from the update kernel; pageable ones take plain copies
        pin = (lambda t: t.pin_memory()) if pinned else (lambda t: t.clone())
        self.h = {}
        for k in PERSISTENT:
            self.h[k] = pin(torch.as_tensor(np.ascontiguousarray(state[k], dtype=np.float64)))
        self.h["id"] = pin(torch.as_tensor(np.ascontiguousarray(state["id"], dtype=np.int64)))
        self.outputs = outputs
        if outputs:
            for k in OUTPUTS:
                self.h[k] = pin(torch.zeros(self.n, dtype=torch.float64))
            self.h["iad"] = pin(torch.zeros(6 * self.n, dtype=torch.float64))
        self.dt = np.zeros(1)
        self._st = SphState()
        for k in _lib.STATE_FIELDS:
            setattr(self._st, k, self.h[k].data_ptr() if k in self.h else None)
        self._st.id = self.h["id"].data_ptr()
        self._st.n = self.n

    def bytes_per_step(self):
        h2d = 8 * (len(PERSISTENT) + 1) * self.n + 8
        d2h = h2d + (8 * (len(OUTPUTS) + 6) * self.n if self.outputs else 0)
        return h2d, d2h

    def step(self):
        with torch.cuda.device(self.device):
            rc = self.lib.sph_step_host(self.ctx, C.byref(self._st),
                                        self.dt.ctypes.data_as(C.c_void_p), _stream_ptr())
        check(self.lib, self.ctx, rc)

    def close(self):
        if getattr(self, "ctx", None):
            with torch.cuda.device(self.device):
                torch.cuda.synchronize()
                self.lib.sph_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
