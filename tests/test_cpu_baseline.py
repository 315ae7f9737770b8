"""The OpenMP CPU baseline (baseline/dem_cpu.cpp) against the FP64 oracle.

The baseline is the program bench.py times on the host cores beside the GPU
library, written in the paper's own design (Sec. 3, Sec. 5).  Its physics
must be the oracle's: after 100 steps of the box pour (1,000 spheres, 12
triangles) and of the turning primitives scene (points, segments, triangles
and rectangles with radii), forces and positions agree to 1e-9 -- its force
sums are accumulated by threads in a timing-dependent order, so the bits
differ, not the values.
"""
import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes


def run_both(oracle_mod, s, steps):
    from baseline import dem_cpu
    V, El, rad = scenes.all_elements(s)
    cs = dem_cpu.CpuScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], V, El, rad)
    cs.step(steps)
    oc = oracle_mod.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], V, El, rad)
    oc.step(steps)
    return cs, oc


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("name", ["box", "primitives_turning"])
def test_cpu_baseline_matches_oracle(oracle_mod, name):
    s = (scenes.box_scene(n=1000, seed=1, speed=0.3) if name == "box"
         else scenes.primitives_scene(omega=20.0))
    cs, oc = run_both(oracle_mod, s, 100)
    F, T = cs.forces()
    Fo, To = oc.forces()
    assert np.abs(Fo).max() > 0
    st, so = cs.state(), oc.state()
    rmin = float(np.min(s["R"]))
    assert rel(F, Fo) <= 1e-9, rel(F, Fo)
    assert rel(T, To) <= 1e-9, rel(T, To)
    assert np.abs(st["x"] - so["x"]).max() / rmin <= 1e-9
    assert rel(st["v"], so["v"]) <= 1e-9
    assert np.abs(st["q"] - so["q"]).max() <= 1e-9


def test_cpu_baseline_reports_its_threads():
    from baseline import dem_cpu
    assert dem_cpu.threads() >= 1
    assert dem_cpu.cpu_model()
