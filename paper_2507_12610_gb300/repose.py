"""The angle-of-repose example (Sec. 5, piling between two plates) on the GPU.

Runs `scenes.repose_scene` until the grains have drained from the bin and the
heap has come to rest, then measures the heap: the angle of repose of both
flanks, mu_eff = tan(theta), the packing fraction of its core, and the
kinetic-energy history of the run.

    python -m paper_2507_12610_gb300.repose --n 20000 --precision mixed
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis, scenes


def run(n=20_000, precision=1, seed=7, max_time=6.0, check=0.02, rest_speed=2e-3,
        skin=0.0, progress=None, **scene_kw) -> dict:
    """Simulate the pile and measure it.  `check` is the physical time between
    state reads (s); the run stops once the mean grain speed stays below
    `rest_speed` (m/s) for three reads in a row with no grain leaving the bin,
    or at max_time."""
    from . import dem
    s = scenes.repose_scene(n=n, seed=seed, **scene_kw)
    p = s["params"]
    dt = p["dt"]
    R = s["R"]
    sc = dem.Scene.from_dict(s, precision=precision, skin=skin)
    k = max(1, int(round(check / dt)))
    hist = []
    calm = 0
    last_bin = None
    t0 = time.perf_counter()
    steps = 0
    while steps * dt < max_time:
        sc.step(k)
        steps += k
        st = sc.state()
        et, er = analysis.kinetic_energy(R, st["v"], st["w"], p["rho"])
        in_bin = int(np.sum(st["x"][:, 2] > s["z_bin"]))
        vmean = float(np.mean(np.linalg.norm(st["v"], axis=1)))
        hist.append((steps * dt, et, er, in_bin, vmean))
        if progress:
            progress(hist[-1])
        calm = calm + 1 if (vmean < rest_speed and in_bin == last_bin) else 0
        last_bin = in_bin
        if calm >= 3:
            break
    wall = time.perf_counter() - t0
    status = sc.synchronize()
    st = sc.state()
    x = st["x"]
    heap = x[:, 2] < s["z_bin"] - 2 * R
    d = 2 * float(R[0])
    ang = analysis.repose_angle(x[heap, 0], x[heap, 2], R[heap], -s["half_floor"],
                                s["half_floor"], 2 * d)
    try:
        phi = analysis.heap_core_fraction(x[heap], R[heap], s["gap"], ang["apex_height"],
                                          ang["apex_x"], ang["mean"], 3 * d)
    except ValueError:
        phi = float("nan")
    return {
        "n": n, "precision": "fp64" if precision == 0 else "mixed", "seed": seed,
        "status": status, "settled": calm >= 3, "t_end": steps * dt, "steps": steps,
        "dt": dt, "wall_s": wall, "particle_steps_per_s": n * steps / wall,
        "heap_grains": int(heap.sum()), "in_bin": hist[-1][3] if hist else n,
        "theta_left": ang["left"], "theta_right": ang["right"], "theta": ang["mean"],
        "mu_eff": math.tan(math.radians(ang["mean"])), "apex_height": ang["apex_height"],
        "packing_core": phi,
        "ke_history": [(round(h[0], 4), h[1], h[2]) for h in hist],
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=20_000)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--max-time", type=float, default=6.0)
    ap.add_argument("--ke", action="store_true", help="keep the kinetic-energy history")
    a = ap.parse_args()
    r = run(a.n, 0 if a.precision == "fp64" else 1, a.seed, a.max_time)
    if not a.ke:
        r.pop("ke_history")
    print(json.dumps(r))


if __name__ == "__main__":
    main()
