"""Pins of the oracle's particle spawning (Sec. 3.1, "Particle generation")."""
import math

import numpy as np

from paper_2507_12610_gb300 import scenes


def _empty(oracle_mod, sp, g=(0.0, 0.0, 0.0), verts=None, elems=None, elem_radius=None):
    p = scenes.base_params(g=g)
    return oracle_mod.OracleScene(p, np.zeros(0), np.zeros((0, 3)), verts=verts, tris=elems,
                                  tri_radius=elem_radius, spawn=sp)


def test_spawn_stream_is_splitmix64(oracle_mod):
    # published first outputs of SplitMix64 from state 0 (Steele, Lea & Flood
    # 2014, reference generator): 0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4,
    # 0x06C45D188009454F; the uniforms are their top 53 bits
    for k, out in enumerate((0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F)):
        assert oracle_mod.spawn_uniform(0, k) == (out >> 11) / 2.0 ** 53


def test_spawned_particles_are_inside_disjoint_and_at_rest(oracle_mod):
    sp = dict(n_max=400, lo=(0, 0, 0), hi=(0.02, 0.02, 0.02), r_min=0.9e-3, r_max=1.1e-3,
              v0=(0, 0, 0), w0=(0, 0, 0), attempts=60, every=1, seed=3)
    oc = _empty(oracle_mod, sp)
    oc.step(10)
    n = oc.active
    assert 100 < n <= 400
    R = oc.radii()
    st = oc.state()
    x = st["x"][:n]
    assert np.all(R[:n] >= 0.9e-3) and np.all(R[:n] <= 1.1e-3) and np.all(R[n:] == 0)
    assert np.all(x >= 0) and np.all(x <= 0.02)
    d = np.linalg.norm(x[:, None] - x[None], axis=-1) + np.eye(n)
    assert np.all(d >= R[:n, None] + R[None, :n])
    # no contacts, no gravity, v0 = w0 = 0: nothing moves or turns
    assert not st["v"][:n].any() and not st["w"][:n].any()
    assert np.all(st["q"][:n] == [1, 0, 0, 0])
    assert len(oc.contacts()[0]) == 0


def test_failed_attempt_carries_its_radius_over(oracle_mod):
    # a box far smaller than a sphere: after the first particle every attempt
    # overlaps it, so the radius drawn by the second attempt is carried over
    # and only the three centre uniforms are drawn per attempt
    seed = 11
    sp = dict(n_max=10, lo=(0, 0, 0), hi=(1e-5, 1e-5, 1e-5), r_min=1e-3, r_max=2e-3,
              v0=(0, 0, 0), w0=(0, 0, 0), attempts=5, every=1, seed=seed)
    oc = _empty(oracle_mod, sp)
    oc.step(1)
    assert oc.active == 1
    assert oc.spawn_draws == 4 + 4 + 3 * 3
    r0 = 1e-3 + oracle_mod.spawn_uniform(seed, 0) * 1e-3
    assert oc.radii()[0] == r0
    # the first particle leaves (v0 along x in the next spawns does not matter):
    # move it away through its own velocity, then the carried radius is used
    oc2 = _empty(oracle_mod, dict(sp, v0=(50.0, 0, 0), every=20))
    oc2.step(20)   # spawn at step 0, particle flies off at 50 m/s
    assert oc2.active == 1
    oc2.step(1)    # event at step 20: the carried radius (draw 4) is placed
    assert oc2.active == 2
    assert oc2.radii()[1] == 1e-3 + oracle_mod.spawn_uniform(seed, 4) * 1e-3


def test_carry_over_keeps_the_radius_distribution_uniform(oracle_mod):
    # dense filling, most attempts fail; small spheres fit more easily, but
    # with the radius carried over the accepted radii stay uniform on
    # [r_min, r_max] (the purpose the paper gives for the carry-over)
    sp = dict(n_max=5000, lo=(0, 0, 0), hi=(0.03, 0.03, 0.03), r_min=0.5e-3, r_max=1.5e-3,
              attempts=400, every=1, seed=5)
    oc = _empty(oracle_mod, sp)
    oc.step(12)
    n = oc.active
    R = oc.radii()[:n]
    assert n > 1000
    # mean of U[0.5, 1.5] mm is 1 mm, sd 0.2887 mm; 4 standard errors
    assert abs(R.mean() - 1e-3) < 4 * 0.2887e-3 / math.sqrt(n)
    # while the fraction of failed attempts is large
    assert oc.spawn_draws > 3 * 12 * 400 * 0.5


def test_spawning_respects_mesh_and_capacity(oracle_mod):
    # the spawn box straddles a floor rectangle of radius 0.5 mm at z = 0
    verts = np.array([[-0.02, -0.02, 0], [0.02, -0.02, 0], [0.02, 0.02, 0], [-0.02, 0.02, 0]])
    elems = np.array([[0, 1, 2, 3]], dtype=np.int32)
    sp = dict(n_max=150, lo=(-0.01, -0.01, -0.002), hi=(0.01, 0.01, 0.004), r_min=1e-3,
              r_max=1e-3, attempts=100, every=1, seed=9)
    oc = _empty(oracle_mod, sp, verts=verts, elems=elems, elem_radius=np.array([0.5e-3]))
    oc.step(30)
    n = oc.active
    assert n == 150
    z = oc.state()["x"][:n, 2]
    assert np.all(np.abs(z) >= 1.5e-3)
