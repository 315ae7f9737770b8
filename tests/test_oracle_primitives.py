"""Pins of the oracle's other mesh primitives (Sec. 3.3): points, segments
and rectangles with a radius R_j >= 0 (rounded edges), next to triangles.
"""
import math

import numpy as np
import pytest

from tests import physics as ph
from tests.test_oracle_pins import E, NU, RHO, params


def _sample_rect(a, b, d, k, rng):
    s, t = rng.uniform(size=(2, k))
    return a + s[:, None] * (b - a) + t[:, None] * (d - a)


def test_closest_point_on_each_primitive_is_the_minimiser(oracle_mod):
    rng = np.random.default_rng(11)
    for _ in range(150):
        p = rng.normal(size=3) * 2
        # point
        a = rng.normal(size=3)
        np.testing.assert_array_equal(oracle_mod.closest_on_element(p, [a]), a)
        # segment
        b = rng.normal(size=3)
        y = oracle_mod.closest_on_element(p, [a, b])
        tt = rng.uniform(size=(3000, 1))
        S = a + tt * (b - a)
        assert np.linalg.norm(S - p, axis=1).min() >= np.linalg.norm(y - p) - 1e-12
        assert np.linalg.norm(np.cross(y - a, b - a)) < 1e-12  # on the line
        # rectangle a, b, c, d with right angles
        u = rng.normal(size=3)
        w = np.cross(u, rng.normal(size=3))
        w *= rng.uniform(0.3, 2.0) / np.linalg.norm(w)
        b, d = a + u, a + w
        c = a + u + w
        y = oracle_mod.closest_on_element(p, [a, b, c, d])
        S = _sample_rect(a, b, d, 4000, rng)
        assert np.linalg.norm(S - p, axis=1).min() >= np.linalg.norm(y - p) - 1e-12
        s_ = np.dot(y - a, u) / np.dot(u, u)
        t_ = np.dot(y - a, w) / np.dot(w, w)
        assert -1e-12 <= s_ <= 1 + 1e-12 and -1e-12 <= t_ <= 1 + 1e-12


def floor(kind, half=0.05):
    V = np.array([[-half, -half, 0], [half, -half, 0], [half, half, 0], [-half, half, 0]], float)
    if kind == "rect":
        return V, np.array([[0, 1, 2, 3]], dtype=np.int32)
    return V, np.array([[0, 1, 2, -1], [0, 2, 3, -1]], dtype=np.int32)


def test_rectangle_floor_equals_triangles_away_from_seam(oracle_mod):
    R, d = 1e-3, 1e-5
    x = np.array([[0.011, -0.017, R - d]])
    v = np.array([[0.05, -0.02, 0.0]])
    w = np.array([[3.0, 1.0, -2.0]])
    out = []
    for kind in ("rect", "tri"):
        V, T = floor(kind)
        sc = oracle_mod.OracleScene(params(), [R], x, v, w, verts=V, tris=T,
                                    tri_radius=np.zeros(len(T)))
        sc.step(1)
        out.append(sc.forces())
    np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-12, atol=0)
    np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-12, atol=1e-30)


def test_rectangle_has_no_ghost_contact_on_the_seam(oracle_mod):
    # Sec. 3.3: rectangles avoid the ghost collision of two coplanar triangles
    # meeting at a seam: on the diagonal the triangle floor pushes twice.
    R, d = 1e-3, 1e-5
    x = np.array([[0.0, 0.0, R - d]])
    forces, keys = {}, {}
    for kind in ("rect", "tri"):
        V, T = floor(kind)
        sc = oracle_mod.OracleScene(params(mu_s=0, mu_r=0, mu_t=0), [R], x, verts=V, tris=T,
                                    tri_radius=np.zeros(len(T)))
        sc.step(1)
        forces[kind] = sc.forces()[0][0, 2]
        keys[kind] = sc.contacts()[0]
    assert len(keys["rect"]) == 1 and len(keys["tri"]) == 2
    assert forces["tri"] == pytest.approx(2 * forces["rect"], rel=1e-12)
    Es = E / (1 - NU ** 2)
    assert forces["rect"] == pytest.approx(4 / 3 * Es * math.sqrt(R) * d ** 1.5, rel=1e-12)


def test_sphere_rests_on_a_rounded_rod_at_the_hertz_overlap(oracle_mod):
    # A segment of radius R_j is a rod with a rounded surface: a sphere resting
    # on it under gravity settles where the wall-limit Hertz force carries its
    # weight, (4/3) E/(1-nu^2) sqrt(R_i) delta^(3/2) = m g (R* = R_i).
    R, Rj = 1e-3, 2e-3
    V = np.array([[-0.05, 0.0, 0.0], [0.05, 0.0, 0.0]])
    T = np.array([[0, 1, -1, -1]], dtype=np.int32)
    m = ph.sphere_mass(RHO, R)
    Es = E / (1 - NU ** 2)
    d_eq = (m * 9.81 / (4 / 3 * Es * math.sqrt(R))) ** (2 / 3)
    x = np.array([[0.003, 0.0, R + Rj - 0.5 * d_eq]])
    p = params(e_n=0.2, mu_s=1.0, mu_r=1.0, mu_t=1.0, g=(0, 0, -9.81), dt=2e-5)
    sc = oracle_mod.OracleScene(p, [R], x, verts=V, tris=T, tri_radius=[Rj])
    sc.step(20000)
    z = sc.state()["x"][0, 2]
    assert R + Rj - z == pytest.approx(d_eq, rel=1e-6)
    assert abs(sc.state()["x"][0, 1]) < 1e-12  # balanced on top, no roll-off


def test_restitution_against_a_point_element(oracle_mod):
    # a point with radius R_j is a fixed sphere of infinite mass: the wall law
    # gives exit/entry speed ratio e_n
    R, Rj, v0, e_n = 1e-3, 0.5e-3, 0.3, 0.5
    m = ph.sphere_mass(RHO, R)
    _, tc = ph.hertz_impact(m, R, E / (1 - NU ** 2), v0)
    dt = tc / 800
    p = params(e_n=e_n, mu_s=0, mu_r=0, mu_t=0, dt=dt)
    V = np.array([[0.0, 0.0, 0.0]])
    T = np.array([[0, -1, -1, -1]], dtype=np.int32)
    sc = oracle_mod.OracleScene(p, [R], [[0, 0, R + Rj + 0.5 * v0 * dt]], [[0, 0, -v0]],
                                verts=V, tris=T, tri_radius=[Rj])
    started = False
    for _ in range(5000):
        sc.step(1)
        if len(sc.contacts()[0]):
            started = True
        elif started:
            break
    assert sc.state()["v"][0, 2] / v0 == pytest.approx(e_n, abs=4e-3)
