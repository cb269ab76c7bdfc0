"""Long run of the rotating square patch (section 4.6) with the conservation
sums tracked every step: total angular momentum L (the quantity the paper
compares between codes), linear momentum and the energies.

    python -m paper_2005_02656_gb300.square_patch --side 100 --t-end 0.5 \\
        --precision fp64 --out patch_L.csv

Each step is one sph_step on the device; the sums of the new state come from
sph_last_diagnostics (one small device-to-host copy per step).  The initial
state is the patch of sph_inputs.square_patch: a cubic lattice on
[-0.5, 0.5]^3, x and y open, z periodic, density 1, u = 1,
v = (omega y, -omega x, 0) with omega = 5 (Eq. 7).
"""
from __future__ import annotations

import argparse
import csv
import time

import numpy as np

FIELDS = ("step", "t", "dt", "Px", "Py", "Pz", "E_kin", "E_int", "Lx", "Ly", "Lz", "nn_min",
          "nn_max")


def run(side: int = 100, t_end: float = 0.5, precision: str = "fp64", max_steps: int = 5000,
        max_seconds: float = 600.0, device: str = "cuda:0", **params):
    """Advances the patch until t >= t_end (or max_steps / max_seconds);
    returns a dict of per-step arrays (index 0 is the initial state), the
    largest smoothing length at the end and the wall time.  Extra keyword
    arguments set Params fields (e.g. ng_target=0 keeps h fixed)."""
    import sph_inputs
    from .sim import Params, SphSim
    s = sph_inputs.square_patch(side)
    prm = Params(box_lo=s["lo"], box_hi=s["hi"], periodic=s["periodic"], precision=precision,
                 angular_sums=1)
    for k, v in params.items():
        setattr(prm, k, v)
    sim = SphSim(s, prm, device=device)
    d0 = sim.diagnostics()
    rows = [[0, 0.0, 0.0, *d0[:8], np.nan, np.nan]]
    t = 0.0
    t0 = time.perf_counter()
    step = 0
    flags = 0
    while t < t_end and step < max_steps and time.perf_counter() - t0 < max_seconds:
        sim.step()
        d = sim.last_diagnostics()
        flags = sim.error_word()
        if flags:
            break  # the step raised a flag (e.g. a singular IAD matrix): its state is not kept
        step += 1
        t += d[8]
        rows.append([step, t, d[8], *d[:8], d[9], d[10]])
    wall = time.perf_counter() - t0
    h_max = float(sim.t["h"].max())
    sim.close()
    arr = np.array(rows, dtype=np.float64)
    out = {k: arr[:, i] for i, k in enumerate(FIELDS)}
    out["wall_s"] = wall
    out["error_flags"] = flags
    out["h_max"] = h_max
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--side", type=int, default=100)
    ap.add_argument("--t-end", type=float, default=0.5)
    ap.add_argument("--precision", choices=["fp64", "fp32_mixed"], default="fp64")
    ap.add_argument("--out", default="square_patch_L.csv")
    ap.add_argument("--adaptive-h", action="store_true",
                    help="adapt h toward 100 neighbours (default: h fixed, see run())")
    a = ap.parse_args(argv)
    r = run(a.side, a.t_end, a.precision, ng_target=100 if a.adaptive_h else 0)
    with open(a.out, "w", newline="") as f:
        w = csv.writer(f)
        w.writerow(FIELDS)
        for i in range(r["t"].shape[0]):
            w.writerow([r[k][i] for k in FIELDS])
    Lz = r["Lz"]
    print(f"{int(r['step'][-1])} steps to t = {r['t'][-1]:.4f} in {r['wall_s']:.2f} s; "
          f"L_z: {Lz[0]:.10e} -> {Lz[-1]:.10e} (relative change {(Lz[-1] - Lz[0]) / abs(Lz[0]):.3e}); "
          f"flags 0x{r['error_flags']:x}")


if __name__ == "__main__":
    main()
