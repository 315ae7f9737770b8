"""The long-run statistics helpers (analysis.py) on inputs with known answers."""
import math

import numpy as np
import pytest

from paper_2507_12610_gb300 import analysis


def test_kinetic_energy_of_solid_spheres():
    R = np.array([1e-3, 2e-3])
    v = np.array([[1.0, 0, 0], [0, 2.0, 0]])
    w = np.array([[0, 0, 10.0], [0, 0, 0]])
    rho = 2500.0
    m = 4 / 3 * math.pi * rho * R ** 3
    et, er = analysis.kinetic_energy(R, v, w, rho)
    assert et == pytest.approx(0.5 * m[0] * 1.0 + 0.5 * m[1] * 4.0, rel=1e-14)
    assert er == pytest.approx(0.5 * 0.4 * m[0] * R[0] ** 2 * 100.0, rel=1e-14)


def test_surface_profile_takes_the_highest_top_per_bin():
    x = np.array([0.05, 0.15, 0.16, 0.35])
    z = np.array([1.0, 2.0, 3.0, 4.0])
    R = np.full(4, 0.5)
    xc, h = analysis.surface_profile(x, z, R, 0.0, 0.4, 0.1)
    np.testing.assert_allclose(xc, [0.05, 0.15, 0.25, 0.35])
    np.testing.assert_allclose(h[[0, 1, 3]], [1.5, 3.5, 4.5])
    assert np.isnan(h[2])


def heap_points(left_deg, right_deg, H=0.05, n=200_000, seed=0):
    # spheres filling a heap with apex at x = 0, height H, flanks of given slopes
    rng = np.random.default_rng(seed)
    L = H / math.tan(math.radians(left_deg))
    Rr = H / math.tan(math.radians(right_deg))
    x = rng.uniform(-L, Rr, n)
    z = rng.uniform(0.0, H, n)
    top = np.where(x < 0, H * (1 + x / L), H * (1 - x / Rr))
    keep = z <= top
    return x[keep], z[keep]


def test_repose_angle_of_an_asymmetric_heap():
    x, z = heap_points(30.0, 40.0)
    R = np.full(x.size, 1e-4)
    ang = analysis.repose_angle(x, z - 1e-4, R, -0.1, 0.1, 1e-3)
    assert ang["left"] == pytest.approx(30.0, abs=0.5)
    assert ang["right"] == pytest.approx(40.0, abs=0.5)
    assert ang["mean"] == pytest.approx(35.0, abs=0.5)
    assert ang["apex_x"] == pytest.approx(0.0, abs=2e-3)


def test_packing_fraction_of_a_simple_cubic_lattice():
    a, r = 2e-3, 1e-3  # touching spheres: pi / 6
    g = np.stack(np.meshgrid(*[np.arange(20)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g + 0.5) * a
    R = np.full(len(x), r)
    phi = analysis.packing_fraction(x, R, (2 * a, 2 * a, 2 * a), (18 * a, 18 * a, 18 * a))
    assert phi == pytest.approx(math.pi / 6, rel=1e-12)


@pytest.mark.parametrize("deg", [-25.0, 30.0, 42.0])
def test_drum_surface_angle_of_a_tilted_bed(deg):
    rng = np.random.default_rng(1)
    Rd, L, n = 0.07, 0.14, 400_000
    x = rng.uniform(-L / 2, L / 2, n)
    y = rng.uniform(-Rd, Rd, n)
    z = rng.uniform(-Rd, Rd, n)
    keep = (np.hypot(y, z) < Rd) & (z < math.tan(math.radians(deg)) * y)
    X = np.stack([x, y, z], 1)[keep]
    R = np.full(len(X), 1e-3)
    got = analysis.drum_surface_angle(X, R, Rd, L, 4e-3)
    assert got == pytest.approx(deg, abs=0.5)


def test_drum_surface_angle_ignores_the_end_caps():
    # spheres piled high near the caps (|x| > L/4) must not change the angle
    rng = np.random.default_rng(2)
    Rd, L, n = 0.07, 0.14, 300_000
    x = rng.uniform(-L / 2, L / 2, n)
    y = rng.uniform(-Rd, Rd, n)
    z = rng.uniform(-Rd, Rd, n)
    slope = math.tan(math.radians(35.0))
    cap = np.abs(x) > 0.3 * L
    keep = (np.hypot(y, z) < Rd) & ((z < slope * y) | (cap & (z < 0.05)))
    X = np.stack([x, y, z], 1)[keep]
    got = analysis.drum_surface_angle(X, np.full(len(X), 1e-3), Rd, L, 4e-3)
    assert got == pytest.approx(35.0, abs=0.5)
