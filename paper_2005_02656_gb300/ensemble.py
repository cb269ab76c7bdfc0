"""Batched ensemble of independent SPH boxes on one GPU (libsph's
sph_ensemble_* entry points): one persistent cooperative launch advances all
boxes by any number of steps; the launch can be captured in a CUDA graph.
PyTorch provides the device memory and the current stream only.
"""
from __future__ import annotations

import ctypes as C
import time

import numpy as np
import torch

from . import _lib
from ._lib import EnsConfig, SphState, check
from .sim import OUTPUTS, PERSISTENT, Params, _stream_ptr


class Ensemble:
    """boxes: list of (state dict from sph_inputs, alpha).  All boxes share the
    physical parameters of `params` except their box geometry and alpha."""

    def __init__(self, boxes, params: Params | None = None, device: str = "cuda:0"):
        self.lib = _lib.load()
        self.device = torch.device(device)
        params = params or Params(precision="fp32_mixed")
        params.precision = "fp32_mixed"
        self.params = params
        self.nbox = len(boxes)
        self.box_n = np.array([b[0]["x"].shape[0] for b in boxes], dtype=np.int64)
        self.p0 = np.concatenate([[0], np.cumsum(self.box_n)[:-1]]).astype(np.int64)
        self.n = int(self.box_n.sum())
        lo = np.array([b[0]["lo"] for b in boxes], dtype=np.float64).ravel()
        hi = np.array([b[0]["hi"] for b in boxes], dtype=np.float64).ravel()
        per = np.array([b[0]["periodic"] for b in boxes], dtype=np.int32).ravel()
        self.alpha = np.array([b[1] for b in boxes], dtype=np.float64)
        cp = params.c()
        self.ctx = C.c_void_p()
        with torch.cuda.device(self.device):
            check(self.lib, None, self.lib.sph_ensemble_init(
                C.byref(cp), self.nbox, self.box_n.ctypes.data_as(C.c_void_p),
                lo.ctypes.data_as(C.c_void_p), hi.ctypes.data_as(C.c_void_p),
                per.ctypes.data_as(C.c_void_p), self.alpha.ctypes.data_as(C.c_void_p),
                C.byref(self.ctx)))
            self.t = {}
            for k in PERSISTENT:
                self.t[k] = torch.as_tensor(
                    np.concatenate([b[0][k] for b in boxes]).astype(np.float64)).to(self.device)
            self.t["id"] = torch.as_tensor(
                np.concatenate([b[0]["id"] for b in boxes]).astype(np.int64)).to(self.device)
            for k in OUTPUTS:
                self.t[k] = torch.zeros(self.n, dtype=torch.float64, device=self.device)
            self.t["iad"] = torch.zeros(6 * self.n, dtype=torch.float64, device=self.device)
            self.t["omega"] = torch.ones(self.n, dtype=torch.float64, device=self.device)
            self.dt = torch.zeros(self.nbox, dtype=torch.float64, device=self.device)
        self.cfg = EnsConfig()
        self.lib.sph_ens_default_config(C.byref(self.cfg))
        self._st = SphState()
        for k in _lib.STATE_FIELDS:
            setattr(self._st, k, self.t[k].data_ptr())
        self._st.id = self.t["id"].data_ptr()
        self._st.n = self.n

    def _err(self, rc):
        if rc != _lib.SPH_OK:
            raise _lib.SphError(rc, (self.lib.sph_ensemble_last_error(self.ctx) or b"").decode())

    def set_config(self, cell_factor=None, blocks_per_sm=None, test_skip_block=None,
                   find_window=None, threads_per_particle=None, momentum_threads=None):
        if cell_factor is not None:
            self.cfg.cell_factor = float(cell_factor)
        if blocks_per_sm is not None:
            self.cfg.blocks_per_sm = int(blocks_per_sm)
        if test_skip_block is not None:
            self.cfg.test_skip_block = int(test_skip_block)
        if find_window is not None:
            self.cfg.find_window = int(find_window)
        if threads_per_particle is not None:
            self.cfg.threads_per_particle = int(threads_per_particle)
        if momentum_threads is not None:
            self.cfg.momentum_threads = int(momentum_threads)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_ensemble_set_config(self.ctx, C.byref(self.cfg)))

    def step(self, steps: int = 1):
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_ensemble_step(self.ctx, C.byref(self._st),
                                                 C.c_void_p(self.dt.data_ptr()), int(steps),
                                                 _stream_ptr()))

    def capture(self, steps: int):
        """Capture `steps` steps of all boxes as a CUDA graph (on a side stream)."""
        self._graph_stream = torch.cuda.Stream(device=self.device)
        with torch.cuda.device(self.device):
            torch.cuda.synchronize(self.device)
            self._err(self.lib.sph_ensemble_capture(
                self.ctx, C.byref(self._st), C.c_void_p(self.dt.data_ptr()), int(steps),
                C.c_void_p(self._graph_stream.cuda_stream)))

    def replay(self):
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_ensemble_replay(self.ctx,
                                                   C.c_void_p(self._graph_stream.cuda_stream)))

    def synchronize(self):
        torch.cuda.synchronize(self.device)

    def error_word(self) -> int:
        f = C.c_uint32(0)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_ensemble_error_word(self.ctx, C.byref(f)))
        return int(f.value)

    def info(self):
        out = np.zeros(4, dtype=np.int64)
        self._err(self.lib.sph_ensemble_info(self.ctx, out.ctypes.data_as(C.c_void_p)))
        return {"particles": int(out[0]), "boxes": int(out[1]), "ctas": int(out[2]),
                "launches": int(out[3])}

    def phase_times(self):
        """Milliseconds per step of each phase since the last call (device
        timer of block 0 between grid barriers), and the step count."""
        ms = np.zeros(len(_lib.ENS_PHASES))
        steps = C.c_int64(0)
        with torch.cuda.device(self.device):
            self._err(self.lib.sph_ensemble_phase_times(self.ctx, ms.ctypes.data_as(C.c_void_p),
                                                         C.byref(steps)))
        k = max(int(steps.value), 1)
        return {name: float(v) / k for name, v in zip(_lib.ENS_PHASES, ms)}, int(steps.value)

    def box_numpy(self, b: int) -> dict:
        """State and outputs of box b, ordered by particle id."""
        torch.cuda.synchronize(self.device)
        lo, hi = int(self.p0[b]), int(self.p0[b] + self.box_n[b])
        out = {k: self.t[k][lo:hi].cpu().numpy() for k in PERSISTENT + OUTPUTS + ("id",)}
        out["iad"] = self.t["iad"][6 * lo:6 * hi].cpu().numpy().reshape(-1, 6)
        order = np.argsort(out["id"], kind="stable")
        return {k: v[order] for k, v in out.items()}

    KNOBS = ("cell_factor", "find_window", "threads_per_particle", "momentum_threads",
             "blocks_per_sm")

    def _time(self, steps, knobs):
        """Seconds per step of `steps` steps of a copy of the current state
        under the configuration `knobs` (the state is restored afterwards)."""
        saved = {k: v.clone() for k, v in self.t.items()}
        saved_dt = self.dt.clone()
        self.set_config(test_skip_block=-1, **knobs)
        self.step(1)                              # warm-up of this configuration
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        self.step(steps)
        torch.cuda.synchronize(self.device)
        sec = (time.perf_counter() - t0) / steps
        for k in self.t:
            self.t[k].copy_(saved[k])
        self.dt.copy_(saved_dt)
        return sec

    def autotune(self, steps: int = 2, cell_factors=(1.0, 1.15, 1.3), find_windows=(128, 256, 512),
                 threads_per_particle=(1, 2, 4), momentum_threads=(4, 2), blocks_per_sm=(0,)):
        """Picks the ensemble kernel's configuration by timing `steps` steps
        of a copy of the current state per candidate: the tile shape of the
        neighbour search (find_window) and the threads per particle of the
        density and IAD phases over their full grid at the first cell factor
        and momentum split, then the momentum split, the cell-size factor and
        the persistent CTAs per SM one at a time around the best.  The
        ensemble's own state is not advanced."""
        results = []

        def trial(**knobs):
            sec = self._time(steps, knobs)
            results.append((sec, dict(knobs)))
            return sec

        best = None
        for w in find_windows:
            for tp in threads_per_particle:
                k = {"cell_factor": cell_factors[0], "find_window": w,
                     "threads_per_particle": tp, "momentum_threads": momentum_threads[0],
                     "blocks_per_sm": blocks_per_sm[0]}
                sec = trial(**k)
                if best is None or sec < best[0]:
                    best = (sec, k)
        for name, values in (("momentum_threads", momentum_threads[1:]),
                             ("cell_factor", cell_factors[1:]), ("blocks_per_sm", blocks_per_sm[1:])):
            for v in values:
                k = dict(best[1], **{name: v})
                sec = trial(**k)
                if sec < best[0]:
                    best = (sec, k)
        self.set_config(test_skip_block=-1, **best[1])
        self.tuning = results
        return dict(best[1], seconds_per_step=best[0],
                    tried=[dict(k, seconds_per_step=s) for s, k in results])

    def close(self):
        if getattr(self, "ctx", None):
            with torch.cuda.device(self.device):
                torch.cuda.synchronize(self.device)
                self.lib.sph_ensemble_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
