"""Checks of the seeded scene generators (inputs only; no method arithmetic)."""
import math

import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes
from tests import physics as ph


@pytest.mark.parametrize("dt,rmin", [(scenes.DT_BOX, 0.9e-3),
                                     (scenes.DT_COLUMN, 1e-3 * math.exp(-0.6)),
                                     (scenes.DT_DRUM, 0.8e-3)])
def test_timesteps_are_one_fiftieth_of_the_hertz_contact_time(dt, rmin):
    # elastic head-on impact of two R_min spheres with peak overlap 10 % of 2R*
    E, nu, rho = 1e6, 0.3, 2500.0
    Rs, ms, Es = rmin / 2, ph.sphere_mass(rho, rmin) / 2, E / (2 * (1 - nu ** 2))
    dmax = 0.1 * 2 * Rs
    v = math.sqrt(16 * Es * math.sqrt(Rs) * dmax ** 2.5 / (15 * ms))
    d_chk, tc = ph.hertz_impact(ms, Rs, Es, v)
    assert d_chk == pytest.approx(dmax, rel=1e-12)
    assert dt == pytest.approx(tc / 50, rel=1e-12)
    # and about a dozen default steps (Eq. dt) per such collision
    assert 11 < tc / (rmin * math.sqrt(rho * (1 - nu ** 2) / E)) < 13


def test_box_scene_is_non_overlapping_and_inside():
    s = scenes.box_scene(n=300, seed=3)
    X, R = s["x"], s["R"]
    lo, hi = s["domain"]
    assert np.all(X - R[:, None] >= lo - 1e-15) and np.all(X + R[:, None] <= hi + 1e-15)
    d = np.linalg.norm(X[:, None] - X[None], axis=-1) + np.eye(len(R)) * 1
    assert np.all(d >= R[:, None] + R[None] - 1e-15)
    assert s["tris"].shape == (12, 3)


def test_drum_mesh_counts_and_closure():
    V, T = scenes.drum_mesh(0.15, 0.3)
    assert T.shape == (4096, 3)
    # closed surface: every edge shared by exactly two triangles
    e = np.sort(np.concatenate([T[:, [0, 1]], T[:, [1, 2]], T[:, [2, 0]]]), axis=1)
    _, cnt = np.unique(e, axis=0, return_counts=True)
    assert np.all(cnt == 2)


def test_drum_scene_fill_and_no_overlap_small():
    s = scenes.drum_scene(n=5000, seed=1)
    X, R = s["x"], s["R"]
    r_in = s["drum_radius"] * math.cos(math.pi / 128)
    assert np.all(np.hypot(X[:, 1], X[:, 2]) + R <= r_in)
    assert np.all(np.abs(X[:, 0]) + R <= 0.5 * s["drum_length"])
    from scipy.spatial import cKDTree
    pairs = cKDTree(X).query_pairs(2.4e-3, output_type="ndarray")
    d = np.linalg.norm(X[pairs[:, 0]] - X[pairs[:, 1]], axis=1)
    assert np.all(d >= R[pairs[:, 0]] + R[pairs[:, 1]])


def test_generators_are_seeded():
    a = scenes.box_scene(n=50, seed=9)
    b = scenes.box_scene(n=50, seed=9)
    np.testing.assert_array_equal(a["x"], b["x"])
    np.testing.assert_array_equal(a["R"], b["R"])


def test_repose_scene_knobs():
    # the sensitivity knobs change only what they name: the time step, the
    # plate gap, the spawn height and the grains' starting speed
    base = scenes.repose_scene(n=20_000)
    assert base["gap"] == pytest.approx(11 * 2e-3)
    assert base["params"]["dt"] == pytest.approx(scenes.eq_dt(1e-3, 1000.0, 0.3, 1e6) / 10)
    fine = scenes.repose_scene(n=20_000, dt_div=20)
    assert fine["params"]["dt"] == pytest.approx(0.5 * base["params"]["dt"])
    assert fine["z_spawn"] == base["z_spawn"] and fine["gap"] == base["gap"]
    wide = scenes.repose_scene(n=20_000, gap_diameters=15)
    assert wide["gap"] == pytest.approx(15 * 2e-3)
    # a wider gap holds the same grains in a lower heap, so the stream starts lower
    assert wide["z_spawn"] < base["z_spawn"]
    low = scenes.repose_scene(n=20_000, spawn_angle=45.0)
    assert low["z_spawn"] < base["z_spawn"] and low["params"]["dt"] == base["params"]["dt"]
    # the spawn box stays above the heap of the named angle
    area = 20_000 * (math.pi / 6.0) * (2e-3) ** 3 / (0.6 * low["gap"])
    assert low["spawn"]["lo"][2] > math.sqrt(area * math.tan(math.radians(45.0)))
    rest = scenes.repose_scene(n=20_000, v0=0.0)
    assert rest["spawn"]["v0"] == (0.0, 0.0, 0.0) and rest["z_spawn"] == base["z_spawn"]
