"""The two smaller standard workloads, run end to end on the GPU.

  box     1,000 spheres (R ~ U[0.9, 1.1] mm) poured into a 20 x 20 x 60 mm box
          of 12 triangles and settling, 10,000 steps;
  column  200,000 spheres (log-normal radii, median 1 mm, sigma 0.2) in a
          free-standing square column of aspect ratio 2 released onto a floor,
          50,000 steps (the granular column collapse).

Each run reports particle-steps/s (wall clock around the steps, after a short
warm-up that builds the step graphs) and a few physical statistics of the end
state, so the two precisions can be compared on them: the kinetic energy and
mean height for the box; for the column the run-out (the 99th percentile of
the spheres' horizontal distance from the axis, relative to the column's half
width) and the final height of the pile relative to the column's.

    python -m paper_2507_12610_gb300.workloads --config column --precision mixed
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import analysis, scenes

CONFIGS = {
    "box": dict(make=lambda n, seed: scenes.box_scene(n=n, seed=seed), n=1000, seed=1,
                steps=10_000),
    "column": dict(make=lambda n, seed: scenes.column_scene(n=n, seed=seed), n=200_000, seed=3,
                   steps=50_000),
}


def run(config: str, precision: int = 1, steps: int | None = None, n: int | None = None,
        seed: int | None = None, warmup: int = 16) -> dict:
    from . import dem
    c = CONFIGS[config]
    n = c["n"] if n is None else n
    seed = c["seed"] if seed is None else seed
    steps = c["steps"] if steps is None else steps
    s = c["make"](n, seed)
    sc = dem.Scene.from_dict(s, precision=precision)
    sc.step(warmup)
    sc.synchronize()
    t0 = time.perf_counter()
    sc.step(steps)
    status = sc.synchronize()
    wall = time.perf_counter() - t0
    st = sc.state()
    stats = sc.stats()
    sc.close()
    R = s["R"]
    et, er = analysis.kinetic_energy(R, st["v"], st["w"], s["params"]["rho"])
    out = {"config": config, "n": n, "seed": seed, "precision": "fp64" if precision == 0 else "mixed",
           "status": status, "steps": steps, "dt": s["params"]["dt"], "wall_s": wall,
           "particle_steps_per_s": n * steps / wall, "rebuilds": stats["rebuilds"],
           "pair_contacts": stats["pair_contacts"], "ke_trans": et, "ke_rot": er}
    x = st["x"]
    if config == "box":
        out["mean_height"] = float(np.mean(x[:, 2]))
    else:
        x0 = s["x"]
        half0 = float(np.max(np.abs(x0[:, :2])))
        h0 = float(np.max(x0[:, 2] + R))
        r = np.hypot(x[:, 0], x[:, 1])
        out["runout"] = float(np.percentile(r, 99.0)) / half0
        out["height"] = float(np.percentile(x[:, 2] + R, 99.9)) / h0
    return out


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--config", choices=sorted(CONFIGS), default="column")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--seed", type=int, default=None)
    a = ap.parse_args()
    print(json.dumps(run(a.config, 0 if a.precision == "fp64" else 1, a.steps, a.n, a.seed)))


if __name__ == "__main__":
    main()
