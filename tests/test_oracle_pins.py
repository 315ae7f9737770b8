"""Pins of the FP64 oracle against what the paper and mechanics fix.

Each test checks the oracle against something other than itself: closed forms
printed in arXiv 2507.12610 (Sec. 2.2 simplified same-material forms and wall
limits), the paper's statements (e_n is the normal velocity ratio; a dozen
steps at Eq. dt; static friction allows equilibrium; symplecticity with
dissipation off), textbook mechanics (Hertz impact, uniformly decelerated
rolling and spinning, discrete free fall, exact rotation composition) and
conservation laws.  A dropped term, a wrong sign or a transposed operand in
the oracle fails at least one of them.
"""
import math

import numpy as np
import pytest

from tests import physics as ph

E, NU, RHO = 1.0e6, 0.3, 2500.0


def params(**over):
    p = dict(E=E, nu=NU, rho=RHO, e_n=0.5, mu_s=0.5, mu_r=0.1, mu_t=0.1, eta=0.0,
             g=(0.0, 0.0, 0.0), dt=1e-5, mesh_omega=(0, 0, 0), mesh_center=(0, 0, 0))
    p.update(over)
    return p


def plane_mesh(half=0.05, z=0.0):
    V = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]])
    T = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    return V, T, np.zeros(2)


# --- Sec. 2.2: effective properties, same-material forms and wall limits -----

@pytest.mark.parametrize("nu", [-0.9, -0.5, 0.0, 0.3, 0.5])
def test_effective_properties_match_printed_same_material_forms(oracle_mod, nu):
    rng = np.random.default_rng(0)
    p = params(nu=nu)
    for _ in range(20):
        Ri, Rj = rng.uniform(0.5e-3, 2e-3, size=2)
        delta = rng.uniform(1e-7, 1e-4)
        c = oracle_mod.contact_coeffs(p, Ri, Rj, delta)
        assert c["Es"] == pytest.approx(E / (2 * (1 - nu ** 2)), rel=1e-14)
        assert c["Gs"] == pytest.approx(E / (4 * (2 - nu) * (1 + nu)), rel=1e-14)
        assert c["ms"] == pytest.approx(4 / 3 * math.pi * RHO / (Ri ** -3 + Rj ** -3), rel=1e-13)
        assert c["Rs"] == pytest.approx(Ri * Rj / (Ri + Rj), rel=1e-14)
        ratio = c["cs"] / c["cn"]
        assert ratio == pytest.approx(math.sqrt((1 - nu) / (10 * (2 - nu))), rel=1e-13)
        assert 0.18 < ratio < 0.26  # range stated for nu in (-1, 0.5]
        # wall limits: R_j = E_j = m_j = infinity
        cw = oracle_mod.contact_coeffs(p, Ri, 0.0, delta, wall=True)
        G = E / (2 * (1 + nu))
        assert cw["Es"] == pytest.approx(E / (1 - nu ** 2), rel=1e-14)
        assert cw["Gs"] == pytest.approx(G / (2 - nu), rel=1e-14)
        assert cw["Rs"] == Ri
        assert cw["ms"] == pytest.approx(ph.sphere_mass(RHO, Ri), rel=1e-14)


# --- normal law: restitution, Hertz impact, "a dozen steps" ------------------

def head_on(oracle_mod, e_n, v0, dt, R=1e-3, wall=False, max_steps=20000):
    """Head-on impact along x; returns (restitution, steps in contact, peak overlap)."""
    p = params(e_n=e_n, mu_s=0.0, mu_r=0.0, mu_t=0.0, dt=dt)
    if wall:
        # sphere moving in -z onto the plane z = 0
        V, T, Rt = plane_mesh()
        x = np.array([[0.011, -0.017, R + 0.5 * v0 * dt]])  # off the diagonal seam
        v = np.array([[0.0, 0.0, -v0]])
        sc = oracle_mod.OracleScene(p, [R], x, v, verts=V, tris=T, tri_radius=Rt)
    else:
        x = np.array([[-R - 0.25 * v0 * dt, 0, 0], [R + 0.25 * v0 * dt, 0, 0]])
        v = np.array([[0.5 * v0, 0, 0], [-0.5 * v0, 0, 0]])
        sc = oracle_mod.OracleScene(p, [R, R], x, v)
    in_contact, started, peak = 0, False, 0.0
    for _ in range(max_steps):
        sc.step(1)
        k, _ = sc.contacts()
        s = sc.state()
        if wall:
            delta = R - s["x"][0, 2]
        else:
            delta = 2 * R - (s["x"][1, 0] - s["x"][0, 0])
        if len(k):
            started = True
            in_contact += 1
            peak = max(peak, delta)
        elif started:
            break
    s = sc.state()
    if wall:
        e = s["v"][0, 2] / v0
    else:
        e = (s["v"][1, 0] - s["v"][0, 0]) / v0
    return e, in_contact, peak


@pytest.mark.parametrize("e_n", [0.1, 0.5, 0.9])
@pytest.mark.parametrize("v0", [0.02, 0.2, 2.0])
def test_restitution_equals_e_n_at_any_speed(oracle_mod, e_n, v0):
    # Sec. 2.2: e_n is the ratio of normal velocities after and before contact.
    # The Hertzian damping law is scale invariant, so this holds at any impact
    # speed; the only error is the O(dt) time discretisation.
    R = 1e-3
    m = ph.sphere_mass(RHO, R)
    _, tc = ph.hertz_impact(m / 2, R / 2, E / (2 * (1 - NU ** 2)), v0)
    e1, _, _ = head_on(oracle_mod, e_n, v0, tc / 400)
    e2, _, _ = head_on(oracle_mod, e_n, v0, tc / 800)
    assert abs(e2 - e_n) < 4e-3
    assert abs(e2 - e_n) < abs(e1 - e_n) or abs(e2 - e_n) < 2e-4  # converges with dt


def test_restitution_against_wall(oracle_mod):
    R, v0, e_n = 1e-3, 0.3, 0.5
    m = ph.sphere_mass(RHO, R)
    _, tc = ph.hertz_impact(m, R, E / (1 - NU ** 2), v0)
    e, _, _ = head_on(oracle_mod, e_n, v0, tc / 800, wall=True)
    assert abs(e - e_n) < 4e-3


@pytest.mark.parametrize("wall", [False, True])
def test_elastic_impact_matches_hertz_closed_form(oracle_mod, wall):
    R, v0 = 1e-3, 0.5
    m = ph.sphere_mass(RHO, R)
    if wall:
        dmax, tc = ph.hertz_impact(m, R, E / (1 - NU ** 2), v0)
    else:
        dmax, tc = ph.hertz_impact(m / 2, R / 2, E / (2 * (1 - NU ** 2)), v0)
    dt = tc / 1000
    e, steps, peak = head_on(oracle_mod, 1.0, v0, dt, wall=wall)
    assert e == pytest.approx(1.0, abs=2e-3)
    assert steps * dt == pytest.approx(tc, rel=3e-3)
    assert peak == pytest.approx(dmax, rel=3e-3)


def test_dozen_steps_at_default_timestep(oracle_mod):
    # Sec. 2.3: Eq. dt resolves a head-on collision of two equal particles with
    # peak relative indentation delta/(2R*) = 10 % in about a dozen steps at
    # e_n = 1/2.  Find the impact speed giving 10 % peak indentation at a fine
    # step, then count steps in contact at Eq. dt.
    R = 1e-3
    dt_eq = R * math.sqrt(RHO * (1 - NU ** 2) / E)
    target = 0.1 * 2 * (R / 2)
    lo, hi = 0.05, 5.0
    for _ in range(30):
        mid = math.sqrt(lo * hi)
        _, _, peak = head_on(oracle_mod, 0.5, mid, dt_eq / 200)
        lo, hi = (mid, hi) if peak < target else (lo, mid)
    _, steps, _ = head_on(oracle_mod, 0.5, math.sqrt(lo * hi), dt_eq)
    assert 10 <= steps <= 14


# --- friction: static hold on an incline, kinetic roll and twist decay -------

def resting_sphere(oracle_mod, theta, mu_s, mu_r, mu_t, R=1e-3, steps=6000, dt=2e-5,
                   w0=(0, 0, 0), v0=(0, 0, 0), g=9.81, e_n=0.5):
    """Sphere on the plane z = 0 with gravity tilted by theta about y."""
    gv = (g * math.sin(theta), 0.0, -g * math.cos(theta))
    p = params(e_n=e_n, mu_s=mu_s, mu_r=mu_r, mu_t=mu_t, dt=dt, g=gv)
    m = ph.sphere_mass(RHO, R)
    Es = E / (1 - NU ** 2)
    N = m * g * math.cos(theta)
    d_eq = (N / (4 / 3 * Es * math.sqrt(R))) ** (2 / 3)
    V, T, Rt = plane_mesh(0.5)
    x0 = np.array([[0.011, -0.017, R - d_eq]])  # off the diagonal seam of the plane
    sc = oracle_mod.OracleScene(p, [R], x0, np.array([v0]), np.array([w0]), verts=V, tris=T,
                                tri_radius=Rt)
    return sc, x0, d_eq


@pytest.mark.parametrize("factor,moves", [(0.8, False), (1.2, True)])
def test_static_sliding_friction_holds_below_tan_mu(oracle_mod, factor, moves):
    mu_s = 0.3
    theta = math.atan(mu_s) * factor
    sc, x0, _ = resting_sphere(oracle_mod, theta, mu_s, 5.0, 5.0)
    sc.step(5000)  # 0.1 s
    s = sc.state()
    disp = s["x"][0, 0] - x0[0, 0]
    if moves:
        # kinetic sliding (rotation held by the strong rolling spring)
        a = 9.81 * (math.sin(theta) - mu_s * math.cos(theta))
        sc.step(2000)
        s2 = sc.state()
        a_num = (s2["v"][0, 0] - s["v"][0, 0]) / (2000 * 2e-5)
        assert a_num == pytest.approx(a, rel=0.01)
    else:
        # bounded static spring deflection, no creep, at rest
        assert abs(disp) < 1e-2 * 1e-3
        sc.step(5000)
        s2 = sc.state()
        assert abs(s2["x"][0, 0] - s["x"][0, 0]) < 1e-9
        assert abs(s2["v"][0, 0]) < 1e-6


@pytest.mark.parametrize("factor,moves", [(0.8, False), (1.2, True)])
def test_rolling_friction_holds_below_its_limit(oracle_mod, factor, moves):
    # Torque balance of a resting sphere: R*|f_r| = r_i |f_s|, so the rolling
    # spring holds while tan(theta) <= mu_r R / r_i (with mu_s large enough).
    mu_r, R = 0.1, 1e-3
    sc, x0, d_eq = resting_sphere(oracle_mod, 0.0, 0.5, mu_r, 5.0)  # to get d_eq at theta=0
    r_i = R - d_eq / 2
    theta = math.atan(mu_r * R / r_i) * factor
    sc, x0, d_eq = resting_sphere(oracle_mod, theta, 0.5, mu_r, 5.0)
    sc.step(5000)
    s = sc.state()
    disp = s["x"][0, 0] - x0[0, 0]
    if moves:
        # once the rolling spring has reached its Coulomb bound: rolling without
        # slipping against kinetic rolling resistance,
        # a = g (sin th - mu_r cos th R / r_i) / (1 + I / (m r_i^2)), I = 2/5 m R^2
        r_i = R - d_eq / 2
        a = 9.81 * (math.sin(theta) - mu_r * math.cos(theta) * R / r_i) / (
            1 + 0.4 * R * R / (r_i * r_i))
        sc.step(2000)
        s2 = sc.state()
        a_num = (s2["v"][0, 0] - s["v"][0, 0]) / (2000 * 2e-5)
        assert a_num == pytest.approx(a, rel=0.02)
        assert s2["w"][0, 1] * r_i == pytest.approx(s2["v"][0, 0], rel=1e-3)  # no slip
    else:
        assert abs(disp) < 1e-2 * R
        sc.step(5000)
        s2 = sc.state()
        assert abs(s2["x"][0, 0] - s["x"][0, 0]) < 1e-9
        assert abs(s2["w"][0, 1]) < 1e-3


def test_twist_decays_uniformly_at_kinetic_rate(oracle_mod):
    # Kinetic twisting torque mu_t |f_n| R* with R* = R for a wall, so a sphere
    # spinning about the floor normal decelerates at 2.5 mu_t g / R.
    R, mu_t, w0 = 1e-3, 0.1, 30.0
    sc, _, _ = resting_sphere(oracle_mod, 0.0, 0.5, 0.1, mu_t, w0=(0, 0, w0), steps=0)
    rate = 2.5 * mu_t * 9.81 / R
    dt = 2e-5
    sc.step(100)  # let the normal contact settle
    w_a = sc.state()["w"][0, 2]
    sc.step(500)
    w_b = sc.state()["w"][0, 2]
    # the static/kinetic alternation of the twist spring lowers the mean
    # torque by O(c_t alpha dt / (mu_t |f_n|)), about 0.6 % here
    assert (w_a - w_b) / (500 * dt) == pytest.approx(rate, rel=1.5e-2)
    sc.step(int(w0 / rate / dt))
    assert abs(sc.state()["w"][0, 2]) < 0.02 * w0


def test_roll_decays_uniformly_at_kinetic_rate(oracle_mod):
    # Rolling on a level floor against kinetic rolling resistance mu_r |f_n|:
    # a = g mu_r (R / r_i) / (1 + I / (m r_i^2)) ~ (5/7) mu_r g.
    R, mu_r, v0 = 1e-3, 0.1, 0.1
    sc0, _, d_eq = resting_sphere(oracle_mod, 0.0, 0.5, mu_r, 5.0)
    r_i = R - d_eq / 2
    sc, _, _ = resting_sphere(oracle_mod, 0.0, 0.5, mu_r, 5.0, v0=(v0, 0, 0),
                              w0=(0, v0 / r_i, 0))
    dt = 2e-5
    sc.step(200)
    va = sc.state()["v"][0, 0]
    sc.step(2000)
    vb = sc.state()["v"][0, 0]
    a = 9.81 * mu_r * (R / r_i) / (1 + 0.4 * R * R / (r_i * r_i))
    assert (va - vb) / (2000 * dt) == pytest.approx(a, rel=2e-2)


# --- conservation laws --------------------------------------------------------

def cluster(oracle_mod, seed=0, n_side=4, spacing=1.9e-3, **over):
    rng = np.random.default_rng(seed)
    g = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = g * spacing + rng.uniform(-5e-5, 5e-5, size=g.shape)
    n = len(x)
    R = rng.uniform(0.9e-3, 1.1e-3, size=n)
    v = rng.normal(scale=0.05, size=(n, 3))
    w = rng.normal(scale=50.0, size=(n, 3))
    p = params(**over)
    return oracle_mod.OracleScene(p, R, x, v, w), R


def test_momentum_and_angular_momentum_conserved_with_friction(oracle_mod):
    sc, R = cluster(oracle_mod, e_n=0.3, mu_s=0.5, mu_r=0.2, mu_t=0.2)
    s0 = sc.state()
    P0 = ph.linear_momentum(RHO, R, s0["v"])
    L0 = ph.angular_momentum(RHO, R, s0["x"], s0["v"], s0["w"])
    m = ph.sphere_mass(RHO, R)
    pscale = (m[:, None] * np.abs(s0["v"])).sum()
    lscale = (m * np.linalg.norm(s0["x"], axis=1) * np.linalg.norm(s0["v"], axis=1)).sum() + (
        0.4 * m * R ** 2 * np.linalg.norm(s0["w"], axis=1)).sum()
    seen = 0
    for _ in range(30):
        sc.step(10)
        seen = max(seen, len(sc.contacts()[0]))
    assert seen > 20
    s1 = sc.state()
    P1 = ph.linear_momentum(RHO, R, s1["v"])
    L1 = ph.angular_momentum(RHO, R, s1["x"], s1["v"], s1["w"])
    assert np.abs(P1 - P0).max() < 1e-13 * pscale
    assert np.abs(L1 - L0).max() < 1e-12 * lscale


def elastic_energy(R, x, Es_pair, Es_wall, lo, hi):
    """Hertz potential (8/15) E* sqrt(R*) delta^(5/2) over touching pairs and walls."""
    n = len(R)
    Epot = 0.0
    for i in range(n):
        d = np.linalg.norm(x[i + 1:] - x[i], axis=1)
        delta = R[i] + R[i + 1:] - d
        Rs = R[i] * R[i + 1:] / (R[i] + R[i + 1:])
        t = delta > 0
        Epot += (8 / 15 * Es_pair * np.sqrt(Rs[t]) * delta[t] ** 2.5).sum()
        for ax in range(3):
            for dw in (x[i, ax] - lo[ax], hi[ax] - x[i, ax]):
                dl = R[i] - dw
                if dl > 0:
                    Epot += 8 / 15 * Es_wall * math.sqrt(R[i]) * dl ** 2.5
    return Epot


def test_energy_bounded_without_dissipation(oracle_mod):
    # Sec. 2.3: with e_n = 1 and mu = eta = 0 the semi-implicit Euler scheme is
    # symplectic: the total energy oscillates at O(dt) but does not drift.
    from paper_2507_12610_gb300 import scenes
    rng = np.random.default_rng(4)
    n_side, sp = 3, 2.05e-3
    g = np.stack(np.meshgrid(*[np.arange(n_side)] * 3, indexing="ij"), -1).reshape(-1, 3)
    x = (g - 1) * sp
    n = len(x)
    R = np.full(n, 1e-3)
    v = rng.normal(scale=0.3, size=(n, 3))
    lo, hi = -np.full(3, 1.6 * sp), np.full(3, 1.6 * sp)
    V, T = scenes.box_mesh(lo, hi)
    m = ph.sphere_mass(RHO, 1e-3)
    _, tc = ph.hertz_impact(m / 2, 0.5e-3, E / (2 * (1 - NU ** 2)), 0.5)
    p = params(e_n=1.0, mu_s=0, mu_r=0, mu_t=0, dt=tc / 50)
    sc = oracle_mod.OracleScene(p, R, x, v, verts=V, tris=T, tri_radius=np.zeros(len(T)))
    Ep, Ew = E / (2 * (1 - NU ** 2)), E / (1 - NU ** 2)
    energies = []
    for _ in range(200):
        sc.step(100)
        s = sc.state()
        energies.append(ph.kinetic_energy(RHO, R, s["v"], s["w"])
                        + elastic_energy(R, s["x"], Ep, Ew, lo, hi))
    e = np.array(energies)
    e0 = ph.kinetic_energy(RHO, R, v, np.zeros_like(v))
    assert np.abs(e - e0).max() < 0.1 * e0  # bounded O(dt) oscillation
    first, last = e[:40].mean(), e[-40:].mean()
    print("energy drift", (last - first) / e0, "max dev", np.abs(e - e0).max() / e0)
    assert abs(last - first) < 0.005 * e0  # no drift


# --- integrator ----------------------------------------------------------------

def test_free_fall_matches_discrete_semi_implicit_euler(oracle_mod):
    # v_n = v0 + n dt g, x_n = x0 + dt sum_{k=1..n} v_k = x0 + n dt v0 + dt^2 g n(n+1)/2;
    # updating x with the old velocity would give n(n-1)/2 instead.
    dt, nsteps = 1e-4, 1000
    g = np.array([0.3, -1.0, -9.81])
    p = params(dt=dt, g=tuple(g))
    x0 = np.array([[0.01, 0.02, 0.03]])
    v0 = np.array([[0.1, 0.0, 0.2]])
    sc = oracle_mod.OracleScene(p, [1e-3], x0, v0)
    sc.step(nsteps)
    s = sc.state()
    n = nsteps
    np.testing.assert_allclose(s["v"][0], v0[0] + n * dt * g, rtol=1e-13, atol=1e-15)
    np.testing.assert_allclose(s["x"][0], x0[0] + n * dt * v0[0] + dt * dt * g * n * (n + 1) / 2,
                               rtol=1e-12, atol=1e-15)


def test_quaternion_free_rotation_composes_exactly(oracle_mod):
    dt, nsteps = 1e-4, 10000
    w = np.array([3.0, -4.0, 12.0])
    q0 = ph.quat_from_axis_angle([1.0, 2.0, 0.5], 0.7)
    sc = oracle_mod.OracleScene(params(dt=dt), [1e-3], [[0, 0, 0]], [[0, 0, 0]], [w], [q0])
    sc.step(nsteps)
    q = sc.state()["q"][0]
    wn = np.linalg.norm(w)
    expect = ph.quat_mul(q0, ph.quat_from_axis_angle(w, nsteps * dt * wn))
    np.testing.assert_allclose(q, expect, atol=2e-12)
    assert abs(np.linalg.norm(q) - 1) < 2e-12  # 1e4 products, each exact to ~1e-16


def test_quaternion_norm_stays_unit_in_collisions(oracle_mod):
    sc, R = cluster(oracle_mod, seed=3, e_n=0.5, mu_s=0.5, mu_r=0.2, mu_t=0.2, dt=2e-5)
    sc.step(2000)
    q = sc.state()["q"]
    assert np.abs(np.linalg.norm(q, axis=1) - 1).max() < 1e-12


# --- contact-point velocity sign (reading of Sec. 2.2) ---------------------------

def spinning_pair(oracle_mod, w_i, w_j, literal):
    R = 1e-3
    x = np.array([[-R + 2e-6, 0, 0], [R - 2e-6, 0, 0]])
    p = params(e_n=0.5, mu_s=0.5, mu_r=0.0, mu_t=0.0, dt=1e-5)
    sc = oracle_mod.OracleScene(p, [R, R], x, np.zeros((2, 3)), np.array([w_i, w_j]),
                                literal_sign=literal)
    return sc


def test_corotating_spheres_slide_and_spin_down(oracle_mod):
    # Equal spheres touching along x, both spinning about +z: their surfaces move
    # in opposite directions at the contact point, so sliding friction must act
    # and slow both spins.  With the printed minus sign the rotational terms
    # cancel and nothing happens, which is unphysical.
    w = (0.0, 0.0, 50.0)
    sc = spinning_pair(oracle_mod, w, w, literal=False)
    sc.step(20)
    _, T = sc.forces()
    assert T[0, 2] < 0 and T[1, 2] < 0
    sc_lit = spinning_pair(oracle_mod, w, w, literal=True)
    sc_lit.step(20)
    _, T_lit = sc_lit.forces()
    assert np.abs(T_lit).max() < 1e-3 * np.abs(T).max()


def test_counter_rotating_spheres_roll_without_sliding(oracle_mod):
    # w_i = -w_j (gear-like): the contact points move together, so there is no
    # sliding force; only rolling resistance (mu_r = 0 here) could act.
    sc = spinning_pair(oracle_mod, (0, 0, 50.0), (0, 0, -50.0), literal=False)
    sc.step(20)
    F, T = sc.forces()
    assert abs(F[0, 1]) < 1e-12 * abs(F[0, 0])
    assert np.abs(T).max() < 1e-12 * abs(F[0, 0]) * 1e-3


# --- contact bookkeeping (Sec. 3.2) and mesh contacts (Sec. 3.3) ---------------

def test_contact_history_created_at_zero_and_dropped_on_separation(oracle_mod):
    R, dt = 1e-3, 1e-6
    vt = 0.05
    x = np.array([[-R - 1e-7, 0, 0], [R + 1e-7, 0, 0]])
    v = np.array([[0.1, vt, 0], [-0.1, 0, 0]])
    p = params(e_n=0.5, mu_s=10.0, mu_r=10.0, mu_t=10.0, dt=dt)
    sc = oracle_mod.OracleScene(p, [R, R], x, v)
    first = None
    seen = 0
    for _ in range(5000):
        sc.step(1)
        k, h = sc.contacts()
        if len(k):
            if first is None:
                first = h[0].copy()
            seen += 1
        elif seen:
            break
    # first contact step: u_s starts at zero and grows by dt times the
    # tangential relative velocity (v_i - v_j has y component vt; w = 0)
    assert first[1] == pytest.approx(dt * vt, rel=1e-3)
    assert abs(first[0]) < 1e-3 * dt * vt
    assert seen > 10 and len(sc.contacts()[0]) == 0


def test_closest_point_on_triangle_is_the_minimiser(oracle_mod):
    rng = np.random.default_rng(7)
    for _ in range(200):
        a, b, c = rng.normal(size=(3, 3))
        p = rng.normal(size=3) * 2
        y = oracle_mod.closest_on_triangle(p, a, b, c)
        # y lies in the triangle
        M = np.stack([b - a, c - a], axis=1)
        st, *_ = np.linalg.lstsq(M, y - a, rcond=None)
        assert np.linalg.norm(a + M @ st - y) < 1e-12
        assert st.min() > -1e-10 and st.sum() < 1 + 1e-10
        # no sampled point of the triangle is closer
        u = rng.uniform(size=(4000, 2))
        u = np.where(u.sum(1, keepdims=True) > 1, 1 - u, u)
        S = a + u[:, :1] * (b - a) + u[:, 1:] * (c - a)
        assert np.linalg.norm(S - p, axis=1).min() >= np.linalg.norm(y - p) - 1e-12


def test_particle_on_shared_edge_touches_both_triangles(oracle_mod):
    # Sec. 3.3: a particle may touch any number of elements; on the seam of two
    # coplanar triangles it is pushed by both (ghost collision kept).
    V, T, Rt = plane_mesh()
    R = 1e-3
    x = np.array([[0.0, 0.0, R - 1e-5]])  # on the diagonal seam of the square
    sc = oracle_mod.OracleScene(params(mu_s=0, mu_r=0, mu_t=0), [R], x, verts=V, tris=T,
                                tri_radius=Rt)
    sc.step(1)
    k, _ = sc.contacts()
    assert sorted(k[:, 1].tolist()) == [-2, -1]
    F, _ = sc.forces()
    Es = E / (1 - NU ** 2)
    assert F[0, 2] == pytest.approx(2 * 4 / 3 * Es * math.sqrt(R) * 1e-5 ** 1.5, rel=1e-12)


def test_rigidly_corotating_particle_feels_only_normal_force(oracle_mod):
    # Rotating mesh reading: wall velocity Omega x (x_c - c) at the contact point
    # and wall angular velocity Omega.  A particle moving rigidly with the mesh
    # has zero relative velocity, so only the elastic normal force acts.
    Om = np.array([0.0, 0.0, 3.0])
    c = np.array([0.01, -0.02, 0.0])
    V, T, Rt = plane_mesh(0.2, z=0.0)
    R, d = 1e-3, 2e-5
    x = np.array([[0.05, 0.03, R - d]])
    v = np.cross(Om, x[0] - c)[None]
    p = params(mesh_omega=tuple(Om), mesh_center=tuple(c), e_n=0.3, mu_s=0.5, mu_r=0.3,
               mu_t=0.3)
    sc = oracle_mod.OracleScene(p, [R], x, v, Om[None], verts=V, tris=T, tri_radius=Rt)
    sc.step(1)
    F, Tq = sc.forces()
    Es = E / (1 - NU ** 2)
    fn = 4 / 3 * Es * math.sqrt(R * d) * d
    assert F[0, 2] == pytest.approx(fn, rel=1e-9)
    assert np.abs(F[0, :2]).max() < 1e-9 * fn
    assert np.abs(Tq).max() < 1e-9 * fn * R


def test_mesh_turns_by_omega_t(oracle_mod):
    # A single triangle rotating about z: after n steps the contact normal of a
    # particle resting on an end face points along the rotated face normal.
    Om = np.array([0.0, 0.0, 2.0])
    dt, nsteps = 1e-4, 2500
    V = np.array([[0.01, -0.01, -0.01], [0.01, 0.01, -0.01], [0.01, 0.0, 0.02]])
    T = np.array([[0, 1, 2]], dtype=np.int32)
    p = params(mesh_omega=tuple(Om), dt=dt, mu_s=0, mu_r=0, mu_t=0, e_n=1.0)
    # particle far away (no contact) just to advance time
    sc = oracle_mod.OracleScene(p, [1e-3], [[1.0, 1.0, 1.0]], verts=V, tris=T,
                                tri_radius=np.zeros(1))
    sc.step(nsteps)
    ang = 2.0 * nsteps * dt
    nrm = np.array([math.cos(ang), math.sin(ang), 0.0])
    # place a probe particle touching the rotated face and step once
    probe_x = 0.01 * nrm + (1e-3 - 1e-5) * nrm
    sc2 = oracle_mod.OracleScene(p, [1e-3], [probe_x], verts=V, tris=T,
                                 tri_radius=np.zeros(1))
    sc2.set_step_count(nsteps)
    sc2.step(1)
    F, _ = sc2.forces()
    assert np.linalg.norm(F[0]) > 0
    np.testing.assert_allclose(F[0] / np.linalg.norm(F[0]), nrm, atol=1e-9)


def test_sampled_first_step_equals_full_step(oracle_mod):
    from paper_2507_12610_gb300 import scenes
    s = scenes.lattice_box_scene((6, 6, 6), spacing=1.95e-3, speed=0.05, spin=20.0)
    sc = oracle_mod.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"],
                                s["verts"], s["tris"], s["tri_radius"])
    sc.step(1)
    F, T = sc.forces()
    st = sc.state()
    ids = np.array([0, 5, 17, 100, 215])
    out = oracle_mod.sample_first_step(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"],
                                       s["verts"], s["tris"], s["tri_radius"], ids)
    np.testing.assert_array_equal(out["F"], F[ids])
    np.testing.assert_array_equal(out["T"], T[ids])
    for k in ("x", "v", "w", "q"):
        np.testing.assert_array_equal(out[k], st[k][ids])


def test_drag_rates_and_spiral_use_pre_update_spin(oracle_mod):
    # Stokes drag (Sec. 2.1): c = 9 eta / (2 rho R^2), gamma = 10/3 c, so a free
    # sphere has v_n = v0 (1 - c dt)^n and w_n = w0 (1 - gamma dt)^n.  With the
    # spin axis fixed, SPIRAL turns by dt|w_k| about w and then by
    # dt^2 |alpha_k| / 2 about alpha = -gamma w_k (the opposite axis), using the
    # spin before its update: total angle = sum_k dt |w_k| (1 - gamma dt / 2).
    eta, R, dt, n = 2e-3, 1e-3, 1e-4, 3000
    c = 9 * eta / (2 * RHO * R * R)
    gam = 10 / 3 * c
    w0 = np.array([0.0, 40.0, 30.0])
    v0 = np.array([0.2, -0.1, 0.05])
    sc = oracle_mod.OracleScene(params(eta=eta, dt=dt), [R], [[0, 0, 0]], [v0], [w0],
                                [[1.0, 0, 0, 0]])
    sc.step(n)
    s = sc.state()
    np.testing.assert_allclose(s["v"][0], v0 * (1 - c * dt) ** n, rtol=1e-12)
    np.testing.assert_allclose(s["w"][0], w0 * (1 - gam * dt) ** n, rtol=1e-12)
    wn = np.linalg.norm(w0)
    angle = dt * wn * (1 - gam * dt / 2) * (1 - (1 - gam * dt) ** n) / (gam * dt)
    np.testing.assert_allclose(s["q"][0], ph.quat_from_axis_angle(w0, angle), atol=1e-12)


def test_spring_projection_keeps_length_worked_example(oracle_mod):
    # Sec. 2.3: the stored spring is projected onto the tangent plane of the
    # current normal and scaled back to its old length.  Sphere at rest on the
    # plane z = 0 (normal +z) with u_s = (3, 0, 4) um stored: it becomes
    # (5, 0, 0) um; static regime and zero relative velocity leave it there.
    R, d = 1e-3, 2e-6
    V, T, Rt = plane_mesh()
    p = params(mu_s=10.0, mu_r=10.0, mu_t=10.0, e_n=0.5)
    sc = oracle_mod.OracleScene(p, [R], [[0.011, -0.017, R - d]], verts=V, tris=T,
                                tri_radius=Rt)
    sc.set_contacts([[0, -1]], [[3e-6, 0, 4e-6, 0, 0, 1e-6, 0.5e-6]])
    sc.step(1)
    k, h = sc.contacts()
    assert k.tolist() == [[0, -1]]
    np.testing.assert_allclose(h[0, :3], [5e-6, 0, 0], rtol=1e-12, atol=1e-20)
    np.testing.assert_allclose(h[0, 3:6], [0, 0, 0], atol=0)  # u_r parallel to n -> zero
    assert h[0, 6] == pytest.approx(0.5e-6, rel=1e-12)  # twisting spring is not projected


def test_kinetic_clip_uses_full_normal_force_including_damping(oracle_mod):
    # Eq. Coulombs bounds |f_s| by mu_s |f_n| with f_n of Eq. fn, which includes
    # the normal dashpot.  On the first step of a fast oblique impact the
    # history is zero and the sliding dashpot alone exceeds the bound, so the
    # sliding force is clipped to exactly mu_s |f_n|: F_t / F_n = -mu_s.
    R, vn, vt, mu = 1e-3, 0.2, 2.0, 0.3
    V, T, Rt = plane_mesh(1.0)
    p = params(e_n=0.5, mu_s=mu, mu_r=0.0, mu_t=0.0, dt=1e-6)
    d0 = 1e-7
    sc = oracle_mod.OracleScene(p, [R], [[0.011, -0.5, R - d0]], [[0, vt, -vn]],
                                verts=V, tris=T, tri_radius=Rt)
    sc.step(1)
    F, _ = sc.forces()
    c = oracle_mod.contact_coeffs(p, R, 0.0, d0, wall=True)
    assert c["cn"] * vn > c["kn"] * d0  # damping dominates the normal force here
    assert F[0, 1] / F[0, 2] == pytest.approx(-mu, rel=1e-12)
    assert F[0, 0] == 0.0


def test_kinetic_reset_with_depth_dependent_stiffness(oracle_mod):
    # The kinetic reset u = -(f + c v) / k of Sec. 2.3 stores the dashpot part in
    # the spring; with k_s and c_s growing with the overlap (Eq. ks), the next
    # step's -k u - c v is no longer the clipped force.  For a fast grazing
    # impact this makes the sliding force change sign during compression, so the
    # net tangential impulse is below the Coulomb-impact value mu (1 + e_n) v_n.
    # This is a property of the method as printed; the test documents it and
    # checks the bound |J_t| <= mu_s * integral |f_n| dt that clipping guarantees.
    R, vn, vt, mu, e_n = 1e-3, 0.2, 2.0, 0.3, 0.5
    m = ph.sphere_mass(RHO, R)
    _, tc = ph.hertz_impact(m, R, E / (1 - NU ** 2), vn)
    dt = tc / 2000
    V, T, Rt = plane_mesh(1.0)
    p = params(e_n=e_n, mu_s=mu, mu_r=0.0, mu_t=0.0, dt=dt)
    sc = oracle_mod.OracleScene(p, [R], [[0.011, -0.5, R + 0.5 * vn * dt]], [[0, vt, -vn]],
                                verts=V, tris=T, tri_radius=Rt)
    started, int_fn, jt = False, 0.0, 0.0
    for _ in range(20000):
        sc.step(1)
        if len(sc.contacts()[0]):
            started = True
            F, _ = sc.forces()
            int_fn += abs(F[0, 2]) * dt
            jt += F[0, 1] * dt
        elif started:
            break
    s = sc.state()
    assert s["v"][0, 2] == pytest.approx(e_n * vn, rel=5e-3)
    assert abs(jt) <= mu * int_fn * (1 + 1e-9)
    assert s["v"][0, 1] - vt == pytest.approx(jt / m, rel=1e-9)


def test_hertzian_damping_gives_e_n_exactly_in_the_continuum():
    # Why the restitution pins can be tight: for the 1-D normal law
    # m* d'' = -k_n(d) d - c_n(d) d' with k_n = 4/3 E* sqrt(R* d) and
    # c_n = beta sqrt(5 m* k_n), the exit/entry speed ratio is e_n itself at
    # any impact speed (solved here by an adaptive ODE integrator, independent
    # of the oracle's time stepping); a damping factor other than sqrt(5) gives
    # a different ratio.
    scipy_integrate = pytest.importorskip("scipy.integrate")
    R, rho = 1e-3, RHO
    Rs, ms, Es = R / 2, ph.sphere_mass(rho, R) / 2, E / (2 * (1 - NU ** 2))

    def ratio(e_n, v0, fac=5.0):
        beta = 1 / math.sqrt(1 + (math.pi / math.log(e_n)) ** 2)

        def f(t, y):
            d = max(y[0], 0.0)
            kn = 4 / 3 * Es * math.sqrt(Rs * d)
            return [y[1], (-kn * y[0] - math.sqrt(fac * ms * kn) * beta * y[1]) / ms]

        ev = lambda t, y: y[0]
        ev.terminal, ev.direction = True, -1
        sol = scipy_integrate.solve_ivp(f, [0, 1], [1e-15, v0], events=ev, rtol=1e-12,
                                        atol=1e-20, max_step=1e-6, method="DOP853")
        return -sol.y_events[0][0][1] / v0

    for e_n in (0.1, 0.5, 0.9):
        for v0 in (0.05, 0.5):
            assert ratio(e_n, v0) == pytest.approx(e_n, abs=1e-8)
    assert abs(ratio(0.5, 0.5, fac=4.0) - 0.5) > 0.02


# --- tangential restitution of the shear dashpot (Sec. 2.2, Eq. cs) ---------

@pytest.mark.parametrize("e_n", [0.2, 0.5, 0.9])
def test_tangential_restitution_of_the_shear_dashpot(oracle_mod, e_n):
    # Sec. 2.2 fixes c_s = sqrt(m* k_s / 6) beta (Eq. cs) and states that it was
    # tuned numerically so that a central collision with the sliding spring
    # held at zero gives e_s = e_n.  With u_s = 0 the tangential contact
    # velocity obeys m_t dv_s/dt = -c_s v_s, where 1/m_t = 1/m_i + 1/m_j +
    # r_i^2/I_i + r_j^2/I_j = 7/(2 m*) for equal solid spheres turning freely
    # (r ~ R); the normal overlap obeys m* delta'' = -k_n delta - c_n delta',
    # and the Hertzian damping of Eq. cn gives ln e_n = -integral c_n dt / (2 m*)
    # over the contact (both damping coefficients scale as delta^(1/4)).  Hence
    # ln e_s = -integral c_s dt / m_t = kappa ln e_n with
    # kappa = (c_s / c_n) (2 m* / m_t) = 7 sqrt((1 - nu) / (10 (2 - nu))),
    # the printed same-material ratio c_s / c_n.  So e_s = e_n^kappa: the
    # claim e_s = e_n would need c_s / c_n = 1/7; with the printed factor
    # kappa = 1.42 at nu = 0.3 (e_s = 0.37 for e_n = 0.5).  The oracle follows
    # the printed equation; this pins its tangential dashpot and the
    # kinematics of its contact velocity to that closed form.
    # a small tangential speed keeps the collision central (the contact normal
    # turns by a negligible angle); the tangential equation is linear, so e_s
    # does not depend on that speed
    # (a slow impact keeps delta << R, so r_i = R_i - delta/2 stays close to R)
    R, v0, vt0 = 1e-3, 0.01, 1e-6
    m = ph.sphere_mass(RHO, R)
    _, tc = ph.hertz_impact(m / 2, R / 2, E / (2 * (1 - NU ** 2)), v0)
    dt = tc / 2000
    big = 1e6  # Coulomb bounds never reached: every step is static
    p = params(e_n=e_n, mu_s=big, mu_r=big, mu_t=big, dt=dt)
    x = np.array([[-R - 0.25 * v0 * dt, 0, 0], [R + 0.25 * v0 * dt, 0, 0]])
    v = np.array([[0.5 * v0, 0.5 * vt0, 0], [-0.5 * v0, -0.5 * vt0, 0]])
    sc = oracle_mod.OracleScene(p, [R, R], x, v)
    started = False
    for _ in range(20000):
        sc.step(1)
        k, h = sc.contacts()
        if len(k):
            started = True
            sc.set_contacts(k, np.zeros_like(h))  # the sliding spring held at zero
        elif started:
            break
    assert started
    s = sc.state()
    d = s["x"][0] - s["x"][1]
    nh = d / np.linalg.norm(d)
    vc = s["v"][0] - s["v"][1] + np.cross(nh, R * s["w"][0] + R * s["w"][1])
    vs = vc - np.dot(vc, nh) * nh
    e_s = float(np.linalg.norm(vs) / vt0)
    e_norm = float(np.dot(s["v"][0] - s["v"][1], nh) / v0)  # separating along nh
    kappa = 7.0 * math.sqrt((1 - NU) / (10 * (2 - NU)))
    assert abs(e_norm - e_n) < 5e-3 * e_n + 1e-3
    assert abs(math.log(e_s) / math.log(e_n) - kappa) < 1e-2 * kappa, (e_s, e_n ** kappa, e_n)
    assert kappa > 1.4 and e_s < e_n  # the printed factor does not give e_s = e_n
