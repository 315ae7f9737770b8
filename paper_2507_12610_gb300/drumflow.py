"""The rotating drum's developed flow, for the statistical comparison of the
two precisions (free-surface angle and kinetic energy).

Runs `scenes.drum_scene` (the benchmark's recipe: an FCC lattice in the lower
part of a closed cylinder turning at 30 rpm about the horizontal x axis) for
a number of revolutions and samples, over the last part of the run, the
angle of the bed's free surface in the middle of the drum and the
translational and rotational kinetic energy.  The drum turns from the start,
so the bed first settles and is lifted until it starts to cascade.

    python -m paper_2507_12610_gb300.drumflow --n 100000 --precision mixed
"""
from __future__ import annotations

import argparse
import json
import math
import time

import numpy as np

from . import analysis, scenes


def run(n=100_000, precision=1, seed=5, revolutions=0.4, sample_from=0.5, sample_dt=0.01,
        skin=0.0, progress=None) -> dict:
    """Simulate `revolutions` turns and sample from the fraction `sample_from`
    of the run on, every `sample_dt` seconds of simulated time."""
    from . import dem
    s = scenes.drum_scene(n=n, seed=seed, nn_dist=2.15e-3, speed=0.02)
    p = s["params"]
    dt = p["dt"]
    om = float(np.linalg.norm(p["mesh_omega"]))
    t_end = revolutions * 2.0 * math.pi / om
    steps_total = int(round(t_end / dt))
    k = max(1, int(round(sample_dt / dt)))
    first = int(round(sample_from * steps_total))
    sc = dem.Scene.from_dict(s, precision=precision, skin=skin)
    R = s["R"]
    d = 2.0 * float(np.max(R))
    t0 = time.perf_counter()
    sc.step(first)
    steps = first
    angles, ke = [], []
    while steps + k <= steps_total:
        sc.step(k)
        steps += k
        st = sc.state()
        angles.append(analysis.drum_surface_angle(st["x"], R, s["drum_radius"],
                                                  s["drum_length"], 2.0 * d))
        et, er = analysis.kinetic_energy(R, st["v"], st["w"], p["rho"])
        ke.append((et, er))
        if progress:
            progress((steps * dt, angles[-1], et, er))
    wall = time.perf_counter() - t0
    status = sc.synchronize()
    sc.close()
    a = np.array(angles)
    e = np.array(ke)
    return {
        "n": n, "precision": "fp64" if precision == 0 else "mixed", "seed": seed,
        "status": status, "steps": steps, "dt": dt, "revolutions": steps * dt * om / (2 * math.pi),
        "samples": len(a), "wall_s": wall, "particle_steps_per_s": n * steps / wall,
        "angle_mean": float(a.mean()), "angle_std": float(a.std()),
        "ke_trans_mean": float(e[:, 0].mean()), "ke_trans_std": float(e[:, 0].std()),
        "ke_rot_mean": float(e[:, 1].mean()), "ke_rot_std": float(e[:, 1].std()),
        "drum_radius": s["drum_radius"],
    }


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--n", type=int, default=100_000)
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="mixed")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--revolutions", type=float, default=0.4)
    ap.add_argument("--sample-from", type=float, default=0.5)
    a = ap.parse_args()
    print(json.dumps(run(a.n, 0 if a.precision == "fp64" else 1, a.seed, a.revolutions,
                         a.sample_from)))


if __name__ == "__main__":
    main()
