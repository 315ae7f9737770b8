"""The angle-of-repose example (Sec. 5, piling between two plates) on the GPU.

Runs `scenes.repose_scene` (a spawned stream of grains between two plates)
until all grains are in and at rest, then measures the heap: the angle of
repose of both flanks, mu_eff = tan(theta), the packing fraction of its core,
and the kinetic-energy history of the run.

    python -m paper_2507_12610_gb300.repose --n 20000 --precision mixed
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis, scenes


def run(n=20_000, precision=1, seed=7, max_time=20.0, check=0.02, rest_speed=2e-3,
        skin=0.0, progress=None, **scene_kw) -> dict:
    """Simulate the pile and measure it.  `check` is the physical time between
    state reads (s); the run stops once all n grains are spawned and their
    mean speed stays below `rest_speed` (m/s) for three reads in a row, or at
    max_time."""
    from . import dem
    s = scenes.repose_scene(n=n, seed=seed, **scene_kw)
    p = s["params"]
    dt = p["dt"]
    R0 = s["spawn"]["r_min"]
    sc = dem.Scene.from_dict(s, precision=precision, skin=skin)
    k = max(1, int(round(check / dt)))
    hist = []
    calm = 0
    t0 = time.perf_counter()
    steps = 0
    while steps * dt < max_time:
        sc.step(k)
        steps += k
        st = sc.state()
        na = sc.active
        R = np.full(n, R0)
        et, er = analysis.kinetic_energy(R[:na], st["v"][:na], st["w"][:na], p["rho"])
        vmean = float(np.mean(np.linalg.norm(st["v"][:na], axis=1))) if na else 0.0
        hist.append((steps * dt, et, er, na, vmean))
        if progress:
            progress(hist[-1])
        calm = calm + 1 if (na == n and vmean < rest_speed) else 0
        if calm >= 3:
            break
    wall = time.perf_counter() - t0
    status = sc.synchronize()
    st = sc.state()
    na = sc.active
    x = st["x"][:na]
    R = np.full(na, R0)
    d = 2 * R0
    ang = analysis.repose_angle(x[:, 0], x[:, 2], R, -s["half_floor"], s["half_floor"], 2 * d)
    try:
        phi = analysis.heap_core_fraction(x, R, s["gap"], ang["apex_height"], ang["apex_x"],
                                          ang["mean"], 3 * d)
    except ValueError:
        phi = float("nan")
    return {
        "n": n, "precision": "fp64" if precision == 0 else "mixed", "seed": seed,
        "status": status, "settled": calm >= 3, "t_end": steps * dt, "steps": steps,
        "dt": dt, "wall_s": wall, "particle_steps_per_s": n * steps / wall, "active": na,
        "theta_left": ang["left"], "theta_right": ang["right"], "theta": ang["mean"],
        "mu_eff": math.tan(math.radians(ang["mean"])), "apex_height": ang["apex_height"],
        "packing_core": phi,
        "ke_history": [(round(h[0], 4), h[1], h[2], h[3]) for h in hist],
    }


def run_many(jobs, workers=None) -> list:
    """Run several heaps at once (a list of keyword dicts for run()), each on a
    CUDA stream of its own from a host thread of its own, so that small heaps
    share the GPU; results in the order of the jobs.  Each heap computes
    exactly what it computes alone."""
    import concurrent.futures as cf

    import torch

    def one(kw):
        with torch.cuda.stream(torch.cuda.Stream()):
            return run(**kw)

    with cf.ThreadPoolExecutor(max_workers=workers or len(jobs)) as ex:
        return list(ex.map(one, jobs))


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=20_000)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--seed", type=int, default=7)
    ap.add_argument("--max-time", type=float, default=20.0)
    ap.add_argument("--ke", action="store_true", help="keep the kinetic-energy history")
    ap.add_argument("--gap", type=float, default=11, help="plate gap in grain diameters")
    ap.add_argument("--dt-div", type=float, default=10.0, help="time step = Eq. dt / this")
    ap.add_argument("--spawn-angle", type=float, default=60.0,
                    help="the spawn box sits above the heap of this angle (deg)")
    ap.add_argument("--v0", type=float, default=-0.5, help="vertical speed of spawned grains")
    a = ap.parse_args()
    r = run(a.n, 0 if a.precision == "fp64" else 1, a.seed, a.max_time, gap_diameters=a.gap,
            dt_div=a.dt_div, spawn_angle=a.spawn_angle, v0=a.v0)
    r.update(gap=a.gap, dt_div=a.dt_div, spawn_angle=a.spawn_angle, v0=a.v0)
    if not a.ke:
        r.pop("ke_history")
    print(json.dumps(r))


if __name__ == "__main__":
    main()
