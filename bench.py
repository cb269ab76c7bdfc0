#!/usr/bin/env python
"""Throughput of one SPH step (the per-step neighbour pipeline of arXiv
2005.02656, section 4) on GB300: particle-updates/s and neighbour-pairs/s,
FP32-mixed (headline) and FP64, on the 8.4M-particle Kelvin-Helmholtz box.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one sph_step: cell grid + Morton sort, neighbour search, density +
EOS, IAD, momentum/energy, global dt, update.  The state and the neighbour
lists (~7 GB) are far larger than L2, so no flush is needed between steps.
Rank 0 prints one JSON line.  Under torchrun each rank advances its own
independent box (replicas: the path has no data exchange between boxes).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import platform
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-updates/s & neighbor-pairs/s per SPH step, FP32-mixed vs FP64, 1 GB300"
UNIT = "particle-updates/s"
KH_NX = 224            # 224x112x112 + 282x141x141 = 8,416,298 particles
SAMPLE_NX = 112        # the same recipe at 1/8 scale for the CPU oracle (1,067,054 particles)

# Flop model per directed neighbour pair (add/sub/mul = 1, FMA = 2,
# rsqrt/div = 1), counted on the operations of each pair loop as written; the
# neighbour search counts per (target, candidate) test.  The FP64 kernels
# evaluate a 15-term series for W (32 flops, 7 terms in FP32) and IAD and
# momentum read W_ab(h_a) cached by the density pass.
FLOPS = {"find": 14, "density": 37, "iad": 57, "momentum": 140}
FLOPS64 = {"find": 14, "density": 43, "iad": 19, "momentum": 131}
# Algorithmic HBM bytes of each kernel launch, every array it touches read or
# written once: per particle (its own fields in and out; the records of
# neighbours counted once, as the particle's own record), per staged slot (the
# 4-byte candidate entry, FP32-mixed), per hit-mask word (8 bytes, FP32-mixed)
# and per list entry (FP32-mixed: the 2-byte staged-slot list; FP64: the int32
# list and the cached W_ab(h_a)).
#   FP32-mixed  find: pos32 16 in, nn 4 out; entries, mask words and slot lists
#               written.  density: rec_d 16, pos32 16, u 8 in; rho, p, c 24,
#               rec_i, recA, recQ 48 out.  IAD: rec_i, recA, recQ 48 in; iad
#               48, recC 16, recC2 8 out.  momentum: recA, recV, recQ, recC,
#               recC2 72 in; ax, ay, az, du 32 out.  Each pass reads the
#               entries and the slot lists once.
#   FP64        find: pos32 16 in, nn 4 out, the list written.  density: x, y,
#               z, h, m, u 48 in, rho, p, c 24 out, the list read and W
#               written.  IAD: x, y, z, h, m, rho 48 in, iad 48 out.  momentum:
#               17 fields 136 in, 32 out; both read the list and W.
KERNEL_BYTES = {
    "fp32_mixed": {"find": {"particle": 20, "slot": 4, "word": 8, "entry": 2},
                   "density": {"particle": 112, "slot": 4, "word": 0, "entry": 2},
                   "iad": {"particle": 120, "slot": 4, "word": 0, "entry": 2},
                   "momentum": {"particle": 104, "slot": 4, "word": 0, "entry": 2}},
    "fp64": {"find": {"particle": 20, "slot": 0, "word": 0, "entry": 4},
             "density": {"particle": 72, "slot": 0, "word": 0, "entry": 12},
             "iad": {"particle": 96, "slot": 0, "word": 0, "entry": 12},
             "momentum": {"particle": 168, "slot": 0, "word": 0, "entry": 12}},
}
# Per particle, the rest of the step (sort and gather 344, dt 16, update 244).
OTHER_BYTES = 604
PAIR_KERNELS = ("find", "density", "iad", "momentum")
# The survey's step model: about 25 kflop and 1.9 KB of HBM traffic per
# particle for the FP32-mixed step at 100 neighbours.
SURVEY_MODEL = {"flops_per_particle": 25_000, "bytes_per_particle": 1_900}
# Derived non-tensor peaks: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz, and
# the FP64 pipe at 1/64 of that rate.
SM, LANES, MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM * LANES * 2 * MHZ * 1e6 / 1e12
FP64_PEAK_TFLOPS = FP32_PEAK_TFLOPS / 64.0
FP32_SRC = "fp32 pipe, derived: 152 SMs x 128 lanes x 2 x 2070 MHz"
FP64_SRC = "fp64 pipe, derived: 1/64 of 152 SMs x 128 lanes x 2 x 2070 MHz"
# DRAM traffic of the pair-path kernels: an ncu capture (dram__bytes_read.sum,
# dram__bytes_write.sum per launch) of the FP32-mixed step on the 1/8-scale KH
# box, committed with the hash of the kernel sources it was taken on.
TRAFFIC_META = os.path.join("profiles", "ncu_dram_kh1m.json")
STAGE_KERNELS = {"find": ("k_find_mask",), "density": ("DensityPass",), "iad": ("IadPass",),
                 "momentum": ("MomentumPass",)}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--nx", type=int, default=KH_NX, help="outer lattice of the KH box")
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-ensemble", action="store_true")
    ap.add_argument("--ensemble-steps", type=int, default=50)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-table", action="store_true", help="skip the lookup-table kernel leg")
    ap.add_argument("--no-gravity", action="store_true", help="skip the self-gravity leg")
    ap.add_argument("--adjoint-side", type=int, default=100)
    ap.add_argument("--pair-mode", choices=["staged", "lists"], default="staged",
                    help="FP32-mixed pair sums: cell-staged candidates with hit masks, or "
                         "int32 neighbour lists")
    return ap.parse_args()


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons.  One sampler runs
    for the whole benchmark (it needs about a second before its first
    sample); each timed region is summarised from the samples inside it."""
    Q = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None
        self.samples = []

    def start(self):
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        import datetime
        if self.p is None:
            return
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(f[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                clk, mxc = float(f[1]), float(f[2])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.NAMES, f[5:9]) if v.lower().startswith("active")}
            self.samples.append((ts, clk, mxc, reasons))

    def summary(self, t0, t1):
        """Samples taken between host times t0 and t1 (0.15 s allowance for
        the sampler's reporting delay)."""
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "samples": 0, "reasons": ["unsampled"]}
        sel = [s for s in self.samples if t0 - 0.15 <= s[0] <= t1 + 0.15]
        reasons = sorted(set().union(*[s[3] for s in sel])) if sel else []
        return {"sm_mhz": statistics.median([s[1] for s in sel]) if sel else None,
                "sm_max_mhz": sel[-1][2] if sel else None, "samples": len(sel),
                "reasons": reasons}


def source_hash(names):
    """Hash of the kernel's source files (a name or a list of names in csrc/)."""
    h = hashlib.sha256()
    for name in ([names] if isinstance(names, str) else names):
        h.update(open(os.path.join(ROOT, "paper_2005_02656_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def read_ncu_csv(path):
    """Per-launch metrics of an `ncu --csv --print-units base` log: a list of
    (launch id, kernel name, {metric: value}) in launch order."""
    import csv
    rows = []
    with open(path, newline="") as f:
        lines = [ln for ln in f if not ln.startswith("==")]
    start = next((i for i, ln in enumerate(lines) if ln.startswith('"ID"')), None)
    if start is None:
        return []
    launches = {}
    for rec in csv.DictReader(lines[start:]):
        try:
            lid = int(rec["ID"])
            val = float(rec["Metric Value"].replace(",", ""))
        except (KeyError, ValueError):
            continue
        unit = rec.get("Metric Unit", "")
        scale = {"byte": 1.0, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "nsecond": 1.0,
                 "usecond": 1e3, "msecond": 1e6}.get(unit, 1.0)
        launches.setdefault(lid, (rec["Kernel Name"], {}))[1][rec["Metric Name"]] = val * scale
    for lid in sorted(launches):
        rows.append((lid, launches[lid][0], launches[lid][1]))
    return rows


def stage_traffic(rows):
    """DRAM bytes (read + write) per stage of the last captured step.  A step
    starts where a search launch follows a launch of another stage; every
    launch of the last step is summed into its stage."""
    def stage_of(name):
        return next((st for st, keys in STAGE_KERNELS.items() if any(k in name for k in keys)),
                    None)
    start, prev = 0, None
    for i, (_, name, _) in enumerate(rows):
        st = stage_of(name)
        if st == "find" and prev != "find":
            start = i
        prev = st
    out = {}
    for _, name, m in rows[start:]:
        st = stage_of(name)
        if st and "dram__bytes_read.sum" in m and "dram__bytes_write.sum" in m:
            out[st] = out.get(st, 0.0) + m["dram__bytes_read.sum"] + m["dram__bytes_write.sum"]
    return out


def traffic_for(stage, n):
    """DRAM bytes per launch of a stage's kernels at n particles, from the
    committed ncu capture scaled by the particle count (the cell populations
    and neighbour counts do not depend on the box size), or None when the
    capture is absent or its kernel sources changed since it was taken."""
    try:
        meta = json.load(open(os.path.join(ROOT, TRAFFIC_META)))
    except Exception:
        return None
    if meta.get("source_sha") != source_hash(meta["source"]):
        return None
    rows = read_ncu_csv(os.path.join(ROOT, "profiles", meta["csv"]))
    b = stage_traffic(rows).get(stage)
    return None if b is None else b * n / meta["n_particles"]


def reduce_max(value, dist, device):
    """Max of a float over the ranks of the process group (identity alone)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_per_rank, world, ms_max):
    """Particle updates per second of all ranks: every rank advances its own
    box of n_per_rank particles; the slowest rank sets the time."""
    return n_per_rank * world / (ms_max * 1e-3)


def conservation(d0, d1, steps):
    """Drift over the timed steps from the sums {Px, Py, Pz, E_kin, E_int, ...}
    before and after them."""
    e0, e1 = d0[3] + d0[4], d1[3] + d1[4]
    return {"energy_rel_change_per_step": (e1 - e0) / abs(e0) / steps,
            "momentum_change": [float(d1[i] - d0[i]) for i in range(3)]}


def run_gpu(args, world, rank, local):
    import numpy as np
    import torch

    import sph_inputs
    from paper_2005_02656_gb300 import HostStepper, Params, SphSim

    dev = f"cuda:{local}"
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        return reduce_max(v, dist, dev)

    clocks = Clocks(local)
    clocks.start()
    windows = {}
    from paper_2005_02656_gb300 import measure_fp32_peak
    fp32_measured = max(measure_fp32_peak() for _ in range(3))   # the FFMA probe, best of 3
    state = sph_inputs.kelvin_helmholtz(args.nx, seed_index=2)
    n = int(state["x"].shape[0])

    def timed(precision, kernel_mode="exact", steps=None, key=None):
        steps = steps or args.steps
        key = key or precision
        sim = SphSim(state, precision=precision, device=dev, kernel_mode=kernel_mode,
                     pair_mode=args.pair_mode)
        stream = torch.cuda.current_stream()
        for _ in range(args.warmup):
            sim.step()
        torch.cuda.synchronize()
        d0 = sim.diagnostics()
        sim.profile(True)
        sim.stage_times()
        st0 = sim.stats()
        l0 = sim.launch_count()
        barrier()
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        tw0 = time.time()
        ev[0].record(stream)
        for i in range(steps):
            sim.step()
            ev[i + 1].record(stream)
        torch.cuda.synchronize()
        tw1 = time.time()
        barrier()
        windows[key] = (tw0, tw1)
        ms = ev[0].elapsed_time(ev[steps]) / steps
        ms_median = statistics.median(ev[i].elapsed_time(ev[i + 1]) for i in range(steps))
        stages, nsteps = sim.stage_times()
        st1 = sim.stats()
        launches = sim.launch_count() - l0
        flags = sim.error_word()
        diag = sim.last_diagnostics()
        d1 = sim.diagnostics()
        sim.close()
        del sim
        torch.cuda.empty_cache()
        pairs = (st1["pairs"] - st0["pairs"]) / steps
        cands = (st1["candidates"] - st0["candidates"]) / steps
        exact = (st1["exact_tests"] - st0["exact_tests"]) / steps
        slots = (st1["staged_slots"] - st0["staged_slots"]) / steps
        words = (st1["mask_words"] - st0["mask_words"]) / steps
        return {"ms": ms, "ms_median": ms_median,
                "stages": {k: v / max(nsteps, 1) for k, v in stages.items()},
                "pairs": pairs, "candidates": cands, "exact_tests": exact, "slots": slots,
                "words": words, "launches": launches,
                "flags": flags, "dt": float(diag[8]),
                "conservation": conservation(d0, d1, steps)}

    r32 = timed("fp32_mixed")
    r64 = None if args.no_fp64 else timed("fp64")
    # the paper's lookup-table kernel (section 4.5) on the same workload
    tab = None
    if not args.no_table:
        tab = {"fp32_mixed": timed("fp32_mixed", "table", steps=5, key="table_fp32_mixed")}
        if not args.no_fp64:
            tab["fp64"] = timed("fp64", "table", steps=3, key="table_fp64")

    e2e = None
    if not args.no_e2e:
        hs = HostStepper(state, Params(box_lo=state["lo"], box_hi=state["hi"],
                                       periodic=state["periodic"], precision="fp32_mixed"),
                         device=dev)
        for _ in range(args.warmup):
            hs.step()
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            hs.step()                      # H2D state, step, D2H new state, sync
        t1 = time.perf_counter()
        barrier()
        h2d, d2h = hs.bytes_per_step()
        hs.close()
        ms_e2e = max_over_ranks((t1 - t0) * 1e3 / args.steps)
        e2e = {"value": whole_job_rate(n, world, ms_e2e), "unit": UNIT, "ms_per_step": ms_e2e,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "path": "sph_step_host (pinned host state, FP32-mixed)"}

    ens = None
    if not args.no_ensemble:
        ens = run_ensemble(args, dev, windows)

    adjoint = None
    if not args.no_adjoint:
        adjoint = run_adjoint(args, dev, windows)

    gravity = None
    if not args.no_gravity:
        gravity = run_gravity(args, dev, windows)

    clocks.stop()
    if ens is not None:
        ens["clocks"] = clocks.summary(*windows["ensemble"])
    if adjoint is not None:
        adjoint["clocks"] = clocks.summary(*windows["adjoint"])
    if gravity is not None:
        for key, r in gravity.items():
            r["clocks"] = clocks.summary(*windows["gravity_" + key])
    for key, r in (("fp32_mixed", r32), ("fp64", r64)):
        if r is not None:
            r["clocks"] = clocks.summary(*windows[key])
    ms32 = max_over_ranks(r32["ms"])
    res = {"n": n, "r32": r32, "r64": r64, "ms32": ms32, "e2e": e2e, "ensemble": ens,
           "fp32_measured": fp32_measured,
           "adjoint": adjoint, "table": tab, "gravity": gravity}
    if r64 is not None:
        res["ms64"] = max_over_ranks(r64["ms"])
    if dist is not None:
        dist.destroy_process_group()
    return res


def run_ensemble(args, dev, windows):
    """Batched ensemble: 256 periodic jittered boxes (sides log-uniform in
    [8, 48], alpha uniform in [0.5, 1.5]), FP32-mixed, autotuned, the given
    number of steps captured as one CUDA graph of one persistent launch."""
    import torch

    import sph_inputs
    from paper_2005_02656_gb300 import Ensemble
    boxes = sph_inputs.ensemble(256)
    ens = Ensemble(boxes, device=dev)
    tune = ens.autotune(steps=2)
    ens.step(3)                                   # warm-up steps of the tuned kernel
    ens.capture(args.ensemble_steps)
    ens.replay()                                  # warm-up replay
    ens.synchronize()
    l0 = ens.info()["launches"]
    ens.phase_times()                             # clears the device phase timer
    stream = ens._graph_stream
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    tw0 = time.time()
    e0.record(stream)
    ens.replay()
    e1.record(stream)
    torch.cuda.synchronize()
    windows["ensemble"] = (tw0, time.time())
    ms = e0.elapsed_time(e1)
    phase_ms, phase_steps = ens.phase_times()
    flags = ens.error_word()
    info = ens.info()
    n = info["particles"]
    ens.close()
    return {"metric": "particle-updates/s, 256-box ensemble, one persistent launch per "
                      f"{args.ensemble_steps}-step CUDA graph", "value": n * args.ensemble_steps / (ms * 1e-3),
            "unit": UNIT, "n_particles": n, "n_boxes": 256, "steps": args.ensemble_steps,
            "ms_per_step": ms / args.ensemble_steps, "gpu_launches": info["launches"] - l0,
            "persistent_ctas": info["ctas"], "error_flags": flags,
            "phase_ms_per_step": {k: round(v, 4) for k, v in phase_ms.items()},
            "phase_steps": phase_steps,
            "autotune": {k: tune[k] for k in ("cell_factor", "find_window", "threads_per_particle",
                                              "momentum_threads",
                                              "blocks_per_sm", "seconds_per_step", "tried")}}


def run_adjoint(args, dev, windows, steps=20, every=5):
    """Gradient of L = sum (rho - 1)^2 + sum m |v|^2 / 2 after 20 FP64 steps
    of the side^3 periodic jittered box (10^6 particles by default) with
    respect to the initial x, v, u and alpha: one forward rollout with a
    checkpoint every 5 steps, one reverse pass (re-running 15 steps from
    checkpoints).  Timed with CUDA events on the current stream after one
    untimed forward + reverse."""
    import torch

    import sph_inputs
    from paper_2005_02656_gb300 import Params, Rollout
    s = sph_inputs.jittered_box(args.adjoint_side, seed_index=3, vel_sigma=0.01)
    n = s["x"].shape[0]
    ro = Rollout(n, steps, every, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"]),
                 device=dev)
    st = {k: torch.as_tensor(s[k], dtype=torch.float64, device=dev)
          for k in ("x", "y", "z", "vx", "vy", "vz", "vxh", "vyh", "vzh", "h", "m", "u",
                    "du_prev")}

    def seed(fin):
        g = torch.zeros_like(fin)
        g[3:6] = st["m"][None, :] * fin[3:6]
        g[7] = 2.0 * (fin[7] - 1.0)
        return g

    fin = ro.forward(st, 1.0)
    ro.backward(seed(fin))
    torch.cuda.synchronize()
    i0 = ro.info()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    tw0 = time.time()
    ev[0].record()
    fin = ro.forward(st, 1.0)
    ev[1].record()
    g = seed(fin)
    gi, ga = ro.backward(g)
    ev[2].record()
    torch.cuda.synchronize()
    windows["adjoint"] = (tw0, time.time())
    i1 = ro.info()
    f_ms, b_ms = ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2])
    finite = bool(torch.isfinite(gi).all()) and bool(torch.isfinite(ga))
    ro.close()
    return {"metric": "particle-steps/s of a full gradient (forward rollout + reverse pass)",
            "value": n * steps / ((f_ms + b_ms) * 1e-3), "unit": "particle-steps/s",
            "workload": f"jittered_box_{n}", "n_particles": n, "steps": steps,
            "checkpoint_every": every, "forward_ms": f_ms, "reverse_ms": b_ms,
            "reverse_over_forward": b_ms / f_ms,
            "recomputed_steps": i1["recomputed_steps"] - i0["recomputed_steps"],
            "gpu_launches": i1["launches"] - i0["launches"], "device_bytes": i1["bytes"],
            "gradient_finite": finite, "dtype": "f64"}


# Operations per interaction of the gravity formulas (add, sub, mul,
# division and square root count 1 each): an accepted node (softened monopole
# + quadrupole) and a particle of an opened leaf.
GRAV_FLOPS = {"node": 65, "particle": 21}


def run_gravity(args, dev, windows, calls=3, theta=0.5):
    """Self-gravity of the about-10^6-particle uniform sphere (open
    boundaries) by the multipole tree, in FP64 and in FP32-mixed: sort, tree
    build, moments and walk per call, timed with CUDA events after one untimed
    call."""
    out = {}
    for precision in ("fp64", "fp32_mixed"):
        out[precision] = _gravity_one(dev, windows, calls, theta, precision)
    return out


def _gravity_one(dev, windows, calls, theta, precision):
    import numpy as np
    import torch

    import sph_inputs
    from paper_2005_02656_gb300 import Params, SphSim
    s = sph_inputs.uniform_sphere(124, seed_index=83)
    n = s["x"].shape[0]
    sim = SphSim(s, Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"],
                           precision=precision), device=dev)
    sim.gravity(1.0, 1e-3, theta)
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    tw0 = time.time()
    ev[0].record()
    counts = np.zeros(2)
    for _ in range(calls):
        _, c = sim.gravity(1.0, 1e-3, theta)
        counts += c
    ev[1].record()
    torch.cuda.synchronize()
    windows["gravity_" + precision] = (tw0, time.time())
    ms = ev[0].elapsed_time(ev[1]) / calls
    flags = sim.error_word()
    sim.close()
    node, part = counts / calls
    flops = GRAV_FLOPS["node"] * node + GRAV_FLOPS["particle"] * part
    achieved = flops / (ms * 1e-3) / 1e12
    if precision == "fp64":
        peak, pk = FP64_PEAK_TFLOPS, "fp64 pipe, derived: 1/64 of 152 SMs x 128 lanes x 2 x 2070 MHz"
    else:
        peak, pk = FP32_PEAK_TFLOPS, "fp32 pipe, derived: 152 SMs x 128 lanes x 2 x 2070 MHz"
    return {"metric": "particles/s of one self-gravity evaluation (tree build + walk)",
            "precision": precision,
            "value": n / (ms * 1e-3), "unit": "particles/s", "workload": f"uniform_sphere_{n}",
            "n_particles": n, "theta": theta, "eps": 1e-3, "ms_per_call": ms,
            "node_interactions": node, "particle_interactions": part,
            "interactions_per_s": (node + part) / (ms * 1e-3), "error_flags": flags,
            "dtype": "f64" if precision == "fp64" else "f32+f64",
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak,
                         "unit": "TFLOP/s", "frac": achieved / peak, "peak_source": pk,
                         "flops_per_call": flops}}


def kernel_bytes(r, n, precision, kern):
    b = KERNEL_BYTES[precision][kern]
    return (b["particle"] * n + b["slot"] * r.get("slots", 0) + b["word"] * r.get("words", 0) +
            b["entry"] * r["pairs"])


def kernel_rooflines(r, n, precision, fp32_measured=None):
    """Each pair-path kernel (search, density, IAD, momentum) against both
    roofs: its flops on the pipe of its precision (derived peak, and the
    probe's measured FP32 rate) and its algorithmic bytes on the measured HBM
    copy bandwidth; `bound` names the nearer roof."""
    hbm = peaks().get("hbm_gbs")
    units = {"find": r["candidates"], "density": r["pairs"], "iad": r["pairs"],
             "momentum": r["pairs"]}
    out = {}
    for k in PAIR_KERNELS:
        ms = r["stages"][k]
        fp64 = precision == "fp64" and k != "find"
        flops = (FLOPS64 if fp64 else FLOPS)[k] * units[k]
        tflops = flops / (ms * 1e-3) / 1e12
        peak = FP64_PEAK_TFLOPS if fp64 else FP32_PEAK_TFLOPS
        alu = {"achieved": tflops, "peak": peak, "unit": "TFLOP/s", "frac": tflops / peak,
               "peak_source": FP64_SRC if fp64 else FP32_SRC, "flops_per_launch": flops}
        if not fp64 and fp32_measured:
            alu["peak_measured"] = fp32_measured
            alu["frac_measured"] = tflops / fp32_measured
        nbytes = kernel_bytes(r, n, precision, k)
        gbs = nbytes / (ms * 1e-3) / 1e9
        mem = {"achieved": gbs, "peak": hbm, "unit": "GB/s", "frac": gbs / hbm if hbm else None,
               "bytes_per_launch": nbytes,
               "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy)" if hbm else None}
        bound = "alu" if mem["frac"] is None or alu["frac"] >= mem["frac"] else "hbm"
        out[k] = {"ms_per_launch": ms, "bound": bound, "alu": alu, "hbm": mem,
                  "traffic": traffic_for(k, n) if precision == "fp32_mixed" else None}
    return out


def step_roofline(r, n, precision, ms_step):
    """The whole step against max(bytes / HBM bandwidth, pipe time of its
    flops): the search on the FP32 pipe, the pair sums on the pipe of the
    path's precision; the kernels run one after another, so pipe times add.
    The survey's model (25 kflop, 1.9 KB per particle, all on the FP32 pipe)
    is given beside it."""
    hbm = peaks().get("hbm_gbs")
    bytes_step = OTHER_BYTES * n + sum(kernel_bytes(r, n, precision, k) for k in PAIR_KERNELS)
    find_ms = FLOPS["find"] * r["candidates"] / (FP32_PEAK_TFLOPS * 1e12) * 1e3
    entries = r["pairs"]
    if precision == "fp64":
        pair_flops = sum(FLOPS64[k] for k in ("density", "iad", "momentum")) * entries
        pair_ms = pair_flops / (FP64_PEAK_TFLOPS * 1e12) * 1e3
    else:
        pair_flops = sum(FLOPS[k] for k in ("density", "iad", "momentum")) * entries
        pair_ms = pair_flops / (FP32_PEAK_TFLOPS * 1e12) * 1e3
    alu_ms = find_ms + pair_ms
    hbm_ms = bytes_step / (hbm * 1e9) * 1e3 if hbm else None
    bound = "alu" if hbm_ms is None or alu_ms >= hbm_ms else "hbm"
    t = max(alu_ms, hbm_ms or 0.0)
    sv_alu = SURVEY_MODEL["flops_per_particle"] * n / (FP32_PEAK_TFLOPS * 1e12) * 1e3
    sv_hbm = SURVEY_MODEL["bytes_per_particle"] * n / (hbm * 1e9) * 1e3 if hbm else None
    sv_t = max(sv_alu, sv_hbm or 0.0)
    return {"bound": bound, "time_ms": t, "alu_ms": alu_ms, "hbm_ms": hbm_ms,
            "frac": t / ms_step, "bytes_per_step": bytes_step,
            "flops_per_step": FLOPS["find"] * r["candidates"] + pair_flops,
            "hbm_peak_gbs": hbm, "peak_source": "HBM: MEASURED_PEAKS.json copy; pipes derived",
            "survey_model": dict(SURVEY_MODEL, alu_ms=sv_alu, hbm_ms=sv_hbm, time_ms=sv_t,
                                 bound="alu" if sv_hbm is None or sv_alu >= sv_hbm else "hbm",
                                 frac=sv_t / ms_step)}


def roofline(r, n, precision, fp32_measured=None):
    """The contract's roofline record: the dominant kernel (longest of the
    four pair-path stages) against its nearer roof."""
    ks = kernel_rooflines(r, n, precision, fp32_measured)
    kern = max(PAIR_KERNELS, key=lambda k: r["stages"][k])
    k = ks[kern]
    roof = k["alu"] if k["bound"] == "alu" else k["hbm"]
    out = {"kernel": f"{kern} ({precision})", "bound": k["bound"], "achieved": roof["achieved"],
           "peak": roof["peak"], "unit": roof["unit"], "frac": roof["frac"],
           "peak_source": roof["peak_source"], "ms_per_launch": k["ms_per_launch"],
           "traffic": k["traffic"]}
    if k["bound"] == "alu":
        out["flops_per_launch"] = roof["flops_per_launch"]
        for key in ("peak_measured", "frac_measured"):
            if key in roof:
                out[key] = roof[key]
    else:
        out["bytes_per_launch"] = roof["bytes_per_launch"]
    return out


def cpu_baseline(max_seconds=20.0, max_steps=5):
    """The FP64 oracle, as it stands, on the host cores: full steps of the KH
    recipe at 1/8 scale, as many as fit in about max_seconds."""
    import numpy as np

    import oracle
    import sph_inputs
    s = sph_inputs.kelvin_helmholtz(SAMPLE_NX, seed_index=2, shuffle=False)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    p = oracle.Params()
    n = s["x"].shape[0]
    dt_prev, steps, t0 = 0.0, 0, time.perf_counter()
    pairs = 0
    while True:
        rc, dt_prev, out = oracle.step(box, s, p, dt_prev)
        steps += 1
        pairs += int(np.asarray(out["nn"]).sum())
        el = time.perf_counter() - t0
        if el >= max_seconds or steps >= max_steps:
            break
    out = {"value": n * steps / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "neighbor_pairs_per_s": pairs / el, "seconds": el,
           "sample": f"{steps} full oracle step(s) of the Kelvin-Helmholtz recipe at 1/8 scale "
                     f"(outer lattice {SAMPLE_NX}, {n} particles), FP64, OpenMP",
           "host": host_cpu()}
    out["small_box"] = oracle_threads_sample()
    out["square_patch"] = oracle_square_patch_sample()
    return out


def oracle_square_patch_sample():
    """One full oracle step of the 10^6-particle rotating square patch (x, y
    open, z periodic) on all cores."""
    import numpy as np

    import oracle
    import sph_inputs
    s = sph_inputs.square_patch(100, shuffle=False)
    n = s["x"].shape[0]
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    t0 = time.perf_counter()
    rc, _, out = oracle.step(box, s, oracle.Params(), 0.0)
    el = time.perf_counter() - t0
    return {"workload": f"square_patch_{n}", "steps": 1, "threads": oracle.num_threads(),
            "value": n / el, "unit": UNIT,
            "neighbor_pairs_per_s": int(np.asarray(out["nn"]).sum()) / el, "rc": rc}


def host_cpu():
    """Core count and CPU model of this host, read at run time."""
    model = None
    try:
        for line in open("/proc/cpuinfo"):
            key = line.split(":")[0].strip().lower()
            if key in ("model name", "cpu model", "hardware"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    if model is None:
        try:
            out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
            for line in out.splitlines():
                if line.lower().startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except Exception:
            pass
    return {"nproc": os.cpu_count(), "model": model, "machine": platform.machine()}


def oracle_threads_sample(steps=3):
    """The oracle on the 8,000-particle periodic box (jittered 20^3 lattice):
    full steps on one thread and on all cores."""
    import numpy as np

    import oracle
    import sph_inputs
    s0 = sph_inputs.jittered_box(20, seed_index=0)
    n = s0["x"].shape[0]
    box = oracle.Box(s0["lo"], s0["hi"], s0["periodic"])
    p = oracle.Params()
    all_cores = oracle.num_threads()
    res = {"workload": f"jittered_box_{n}", "steps": steps}
    for label, threads in (("one_thread", 1), ("all_cores", all_cores)):
        used = oracle.set_num_threads(threads)
        s = {k: (v.copy() if isinstance(v, np.ndarray) else v) for k, v in s0.items()}
        dt_prev, pairs = 0.0, 0
        t0 = time.perf_counter()
        for _ in range(steps):
            rc, dt_prev, out = oracle.step(box, s, p, dt_prev)
            pairs += int(np.asarray(out["nn"]).sum())
        el = time.perf_counter() - t0
        res[label] = {"threads": used, "value": n * steps / el, "unit": UNIT,
                      "neighbor_pairs_per_s": pairs / el}
    oracle.set_num_threads(all_cores)
    return res


def main():
    args = parse()
    world, rank, local = dist_env()
    if args.impl == "reference":
        if rank != 0:
            return 0
        return reference_arm(args, world)
    res = run_gpu(args, world, rank, local)
    if rank != 0:
        return 0
    n = res["n"]
    r32, r64 = res["r32"], res["r64"]
    ms = res["ms32"]
    value = whole_job_rate(n, world, ms)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"kelvin_helmholtz_{n}", "n_particles": n,
                   "box": "[0,1]x[0,1]x[0,0.5] periodic", "precision": "fp32_mixed",
                   "neighbors_target": 100, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "no flush: state + lists ~7 GB >> 129 MB L2"},
        "neighbor_pairs_per_s": r32["pairs"] * world / (ms * 1e-3),
        "ms_per_step_median": r32["ms_median"],
        "stages_ms": r32["stages"],
        "roofline": roofline(r32, n, "fp32_mixed", res["fp32_measured"]),
        "kernels_roofline": kernel_rooflines(r32, n, "fp32_mixed", res["fp32_measured"]),
        "step_roofline": step_roofline(r32, n, "fp32_mixed", ms),
        "fp32_peak": {"derived_tflops": FP32_PEAK_TFLOPS, "measured_tflops": res["fp32_measured"],
                      "measured_by": "sph_measure_fp32_peak: dependent-FMA chains, 8 per thread, "
                                     "8 CTAs of 256 threads per SM, best of 3"},
        "gpu_launches": r32["launches"],
        "clocks": r32["clocks"],
        "error_flags": r32["flags"],
        "conservation": r32["conservation"],
        "search": {"candidates_per_step": r32["candidates"], "exact_tests_per_step": r32["exact_tests"],
                   "pairs_per_step": r32["pairs"], "staged_slots_per_step": r32["slots"],
                   "mask_words_per_step": r32["words"]},
    }
    if r64 is not None:
        ms64 = res["ms64"]
        line["fp64"] = {"value": whole_job_rate(n, world, ms64), "unit": UNIT, "ms_per_step": ms64,
                        "ms_per_step_median": r64["ms_median"],
                        "neighbor_pairs_per_s": r64["pairs"] * world / (ms64 * 1e-3),
                        "stages_ms": r64["stages"], "roofline": roofline(r64, n, "fp64"),
                        "kernels_roofline": kernel_rooflines(r64, n, "fp64"),
                        "step_roofline": step_roofline(r64, n, "fp64", ms64),
                        "gpu_launches": r64["launches"], "error_flags": r64["flags"],
                        "conservation": r64["conservation"], "clocks": r64["clocks"]}
        line["fp32_mixed_over_fp64"] = ms64 / ms
    line["e2e"] = res["e2e"]
    if res.get("ensemble") is not None:
        line["ensemble"] = res["ensemble"]
    if res.get("adjoint") is not None:
        line["adjoint"] = res["adjoint"]
    if res.get("gravity") is not None:
        line["gravity"] = res["gravity"]
    if res.get("table") is not None:
        exact_ms = {"fp32_mixed": ms, "fp64": res.get("ms64")}
        line["kernel_table"] = {
            prec: {"ms_per_step": r["ms"], "stages_ms": r["stages"], "error_flags": r["flags"],
                   "time_vs_exact": (r["ms"] / exact_ms[prec]) if exact_ms.get(prec) else None}
            for prec, r in res["table"].items()}
    if not args.no_cpu and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


def reference_arm(args, world):
    """--impl reference: the FP64 oracle on the host cores, each step a full
    oracle step of the KH recipe at 1/8 scale."""
    import numpy as np

    import oracle
    import sph_inputs
    s = sph_inputs.kelvin_helmholtz(SAMPLE_NX, seed_index=2, shuffle=False)
    box = oracle.Box(s["lo"], s["hi"], s["periodic"])
    p = oracle.Params()
    n = s["x"].shape[0]
    dt_prev = 0.0
    for _ in range(args.warmup):
        rc, dt_prev, _ = oracle.step(box, s, p, dt_prev)
    t0 = time.perf_counter()
    pairs = 0
    for _ in range(args.steps):
        rc, dt_prev, out = oracle.step(box, s, p, dt_prev)
        pairs += int(np.asarray(out["nn"]).sum())
    el = time.perf_counter() - t0
    ms = el * 1e3 / args.steps
    value = n / (ms * 1e-3)
    sample = (f"full oracle steps of the Kelvin-Helmholtz recipe at 1/8 scale "
              f"(outer lattice {SAMPLE_NX}, {n} particles), FP64, OpenMP")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"kelvin_helmholtz_{n}", "n_particles": n,
                       "note": "CPU oracle on a 1/8-scale sample of the GPU arm's workload"},
            "neighbor_pairs_per_s": pairs / el,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
