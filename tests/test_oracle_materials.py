"""Pins of per-particle friction materials in the oracle (batched-scene
extension; the paper has a single material)."""
import math

import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes


def _run(oracle_mod, s, steps, **kw):
    V, El, rad = scenes.all_elements(s)
    oc = oracle_mod.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], V, El, rad,
                                **kw)
    oc.step(steps)
    return oc


def test_one_material_equal_to_the_parameters_is_the_plain_run(oracle_mod):
    s = scenes.box_scene(n=200, seed=2, speed=0.3)
    p = s["params"]
    a = _run(oracle_mod, s, 150)
    b = _run(oracle_mod, s, 150, material=np.zeros(200, dtype=np.int32),
             material_mu=[[p["mu_s"], p["mu_r"], p["mu_t"]]])
    for k in ("x", "v", "w", "q"):
        assert np.array_equal(a.state()[k], b.state()[k]), k
    ka, ha = a.contacts()
    kb, hb = b.contacts()
    assert np.array_equal(ka, kb) and np.array_equal(ha, hb)


@pytest.mark.parametrize("mu_a,mu_b", [(0.2, 0.6), (0.6, 0.2), (0.3, 0.3)])
def test_kinetic_pair_slides_at_the_mean_coefficient(oracle_mod, mu_a, mu_b):
    # two overlapping spheres with a fast tangential relative velocity and no
    # spin: the first-step sliding force is clipped to mean(mu) |f_n| (rolling
    # and twisting springs stay zero)
    R = 1e-3
    x = np.array([[0.0, 0.0, 0.0], [2 * R - 2e-5, 0.0, 0.0]])
    v = np.array([[0.0, 0.5, 0.2], [0.0, -0.5, 0.0]])
    p = scenes.base_params(g=(0.0, 0.0, 0.0), mu_s=0.9)
    oc = oracle_mod.OracleScene(p, [R, R], x, v, material=[0, 1],
                                material_mu=[[mu_a, 0.1, 0.1], [mu_b, 0.1, 0.1]])
    oc.step(1)
    F, _ = oc.forces()
    Fn = F[0, 0]
    Ft = math.hypot(F[0, 1], F[0, 2])
    assert Ft == pytest.approx((mu_a + mu_b) / 2 * abs(Fn), rel=1e-12)


@pytest.mark.parametrize("factor,moves", [(0.8, False), (1.25, True)])
def test_wall_contact_uses_the_particle_material(oracle_mod, factor, moves):
    # the parameters say frictionless; the sphere's material holds it on an
    # incline below tan(theta) = mu_s and lets it slide above
    R, mu_s, g = 1e-3, 0.3, 9.81
    theta = math.atan(mu_s) * factor
    gv = (g * math.sin(theta), 0.0, -g * math.cos(theta))
    p = scenes.base_params(g=gv, mu_s=0.0, mu_r=0.0, mu_t=0.0, dt=2e-5, rho=2500.0)
    Es = 1e6 / (1 - 0.3 ** 2)
    m = 4 / 3 * math.pi * 2500.0 * R ** 3
    d_eq = (m * g * math.cos(theta) / (4 / 3 * Es * math.sqrt(R))) ** (2 / 3)
    V = np.array([[-0.5, -0.5, 0], [0.5, -0.5, 0], [0.5, 0.5, 0], [-0.5, 0.5, 0]])
    x0 = np.array([[0.011, -0.017, R - d_eq]])
    oc = oracle_mod.OracleScene(p, [R], x0, verts=V, tris=np.array([[0, 1, 2, 3]]),
                                tri_radius=[0.0], material=[0], material_mu=[[mu_s, 5.0, 5.0]])
    oc.step(5000)
    disp = oc.state()["x"][0, 0] - x0[0, 0]
    if moves:
        assert disp > 1e-3
    else:
        assert abs(disp) < 1e-5


def test_far_apart_scenes_run_like_separate_runs(oracle_mod):
    # two settling lattices with different materials, 1 m apart, in one run:
    # each behaves as its own run with the material's coefficients (to the
    # rounding of the translated coordinates)
    mus = [(0.2, 0.05, 0.05), (0.7, 0.15, 0.1)]
    parts = []
    for k, mu in enumerate(mus):
        s = scenes.lattice_box_scene((4, 4, 4), seed=3 + k, spacing=1.96e-3, jitter=2e-5,
                                     speed=0.05, walls=False, gravity=False)
        parts.append(s)
    off = np.array([1.0, 0.0, 0.0])
    x = np.vstack([parts[0]["x"], parts[1]["x"] + off])
    R = np.concatenate([parts[0]["R"], parts[1]["R"]])
    v = np.vstack([parts[0]["v"], parts[1]["v"]])
    w = np.vstack([parts[0]["w"], parts[1]["w"]])
    q = np.vstack([parts[0]["q"], parts[1]["q"]])
    n0 = len(parts[0]["R"])
    both = oracle_mod.OracleScene(parts[0]["params"], R, x, v, w, q,
                                  material=[0] * n0 + [1] * (len(R) - n0), material_mu=mus)
    both.step(200)
    st = both.state()
    for k, (s, mu) in enumerate(zip(parts, mus)):
        p = dict(s["params"], mu_s=mu[0], mu_r=mu[1], mu_t=mu[2])
        one = oracle_mod.OracleScene(p, s["R"], s["x"], s["v"], s["w"], s["q"])
        one.step(200)
        sl = slice(0, n0) if k == 0 else slice(n0, None)
        assert np.abs(st["x"][sl] - k * off - one.state()["x"]).max() < 1e-12
        assert np.abs(st["v"][sl] - one.state()["v"]).max() < 1e-9 * np.abs(one.state()["v"]).max()
