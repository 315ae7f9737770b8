"""Parity of the CUDA DEM path (through the C ABI) with the FP64 oracle.

Tolerances (stated by the target of this library): after 100 steps from the
same seeded state, forces and torques of the last step, and the positions,
match the FP64 oracle to a relative 1e-12 in DEM_FP64 and 1e-5 in DEM_MIXED.
Measures:
  forces / torques   max|a - b| / max|b| over the whole array
  positions          max|x - x_ref| / R_min  (coordinates are not a meaningful
                     denominator; R_min is the length scale of the contact law)
  velocities, spins  max|a - b| / max|b|
Contact sets (pair keys) must agree exactly; histories to the same tolerance
relative to the largest history entry.
"""
import math

import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-5}  # DEM_FP64, DEM_MIXED, DEM_MIXED64
PREC_NAME = {0: "fp64", 1: "mixed", 2: "mixed64"}


@pytest.fixture(scope="module")
def dem():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_12610_gb300 import build
    build.build()
    from paper_2507_12610_gb300 import dem as d
    d.load()
    return d


def rel(a, b):
    den = np.abs(b).max()
    return float(np.abs(a - b).max() / den) if den > 0 else float(np.abs(a - b).max())


def oracle_scene(oracle_mod, s):
    V, El, rad = scenes.all_elements(s)
    return oracle_mod.OracleScene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], V, El,
                                  rad)


def run_pair(dem, oracle_mod, s, steps, precision, **kw):
    sc = dem.Scene.from_dict(s, precision=precision, record_forces=True, **kw)
    sc.step(steps)
    assert sc.synchronize() == 0
    oc = oracle_scene(oracle_mod, s)
    oc.step(steps)
    return sc, oc


def compare(sc, oc, s, precision, label=""):
    # the stated bound covers forces, torques and positions; velocities, spins,
    # orientations and spring histories are held to it in DEM_FP64 and to 10x
    # it in DEM_MIXED (FP32 springs accumulate dt v_s in single precision)
    tol = TOL[precision]
    tol_aux = tol if precision == 0 else 10 * tol
    F, T = sc.forces()
    Fo, To = oc.forces()
    st, so = sc.state(), oc.state()
    rmin = float(np.min(s["R"]))
    errs = {
        "F": rel(F, Fo), "T": rel(T, To),
        "x": float(np.abs(st["x"] - so["x"]).max() / rmin),
        "v": rel(st["v"], so["v"]), "w": rel(st["w"], so["w"]),
        "q": float(np.abs(st["q"] - so["q"]).max()),
    }
    k, h = sc.contacts()
    ko, ho = oc.contacts()
    assert np.array_equal(k, ko), f"{label}: contact sets differ ({len(k)} vs {len(ko)})"
    assert len(ko) > 0, f"{label}: scene has no contacts"
    errs["hist"] = rel(h, ho) if len(ho) else 0.0
    bad = {key: val for key, val in errs.items()
           if not val <= (tol if key in ("F", "T", "x") else tol_aux)}
    assert not bad, f"{label}: {bad} (tol {tol}); all {errs}"
    return errs


SCENES = {
    "box_pour": lambda: scenes.box_scene(n=1000, seed=1, speed=0.3),
    "lattice_settling": lambda: scenes.lattice_box_scene((8, 8, 8), seed=2, spacing=1.96e-3,
                                                         jitter=2e-5, speed=0.02),
    "lattice_spinning": lambda: scenes.lattice_box_scene((8, 8, 8), seed=2, spacing=1.96e-3,
                                                         jitter=2e-5, speed=0.05, spin=30.0),
    "drum_small": lambda: scenes.drum_scene(n=1500, seed=4, n_theta=32, n_rings=4,
                                            nn_dist=2.3e-3, radius=0.022),
    "column_2000": lambda: scenes.column_scene(n=2000, seed=3, spacing=2.7e-3),
    # points, segments, triangles, rectangles (Sec. 3.3), resting and turning
    "primitives": lambda: scenes.primitives_scene(),
    "primitives_turning": lambda: scenes.primitives_scene(omega=20.0),
}
# Scenes whose contacts slide, roll and twist at their Coulomb limit for many
# steps.  There the friction update of Sec. 2.3 (Eqs. um_static, fm_kinetic)
# is discontinuous: a static step adds dt v to the spring, a kinetic step does
# not, so a contact whose trial force is within FP32 rounding of mu |f_n| can
# take the other branch in DEM_MIXED, and over a free 100-step run the
# difference of one spring (dt |v|) grows chaotically.  DEM_MIXED is checked on
# these scenes step by step instead (test_mixed_parity_every_step, which runs
# on every scene), and on a settled start where no contact sits at the bound
# (test_free_run_from_settled_column).
COULOMB_LIMIT_SCENES = {"lattice_spinning", "column_2000", "primitives", "primitives_turning"}
CASES = [(name, prec) for name in SCENES for prec in (0, 1, 2)
         if not (prec > 0 and name in COULOMB_LIMIT_SCENES)]


@pytest.mark.parametrize("name,precision", CASES,
                         ids=[f"{n}-{PREC_NAME[p]}" for n, p in CASES])
def test_parity_after_100_steps(dem, oracle_mod, name, precision):
    s = SCENES[name]()
    sc, oc = run_pair(dem, oracle_mod, s, 100, precision)
    compare(sc, oc, s, precision, f"{name}/{precision}")
    if name.startswith("primitives"):
        # the triangle, the inner plate, the capsule and the sphere all touch
        k, _ = sc.contacts()
        touched = set((-1 - k[k[:, 1] < 0, 1]).tolist())
        assert {0, 7, 8, 9} <= touched, touched


# A contact "at the Coulomb bound" has a trial force within this relative band
# of mu |f_n| in the oracle (FP32 evaluates |f| and mu |f_n| to ~1e-7 relative,
# so only such contacts can take the other branch in DEM_MIXED).
COULOMB_BAND = 1e-4
# Branch flips allowed per step (each moves one spring by about dt |v|).
MAX_FLIPS_PER_STEP = 4


def seed_oracle_from(oc, sc):
    """Put the GPU scene's state and friction history into the oracle."""
    st = sc.state()
    oc.set_state(st["x"], st["v"], st["w"], st["q"])
    k, h = sc.contacts()
    oc.set_contacts(k, h)
    oc.set_step_count(sc.stats()["steps"])


@pytest.mark.parametrize("precision", [1, 2], ids=["mixed", "mixed64"])
@pytest.mark.parametrize("name", list(SCENES))
def test_mixed_parity_every_step(dem, oracle_mod, name, precision):
    # DEM_MIXED and the oracle advance together for 100 steps; before every
    # step the oracle takes the GPU's state and friction history (exact in
    # double), so each step is compared from the same start.  Every step:
    # forces and torques within 1e-5 of max|F|, max|T|, positions within
    # 1e-5 R_min, velocities and spins within 1e-4, contact sets identical,
    # springs within 1e-4 of the largest spring -- except at contacts whose
    # oracle trial force sits within COULOMB_BAND of the Coulomb bound, where
    # FP32 may take the other branch (at most MAX_FLIPS_PER_STEP a step).
    s = SCENES[name]()
    sc = dem.Scene.from_dict(s, precision=precision, record_forces=True)
    oc = oracle_scene(oracle_mod, s)
    rmin = float(np.min(s["R"]))
    worst = {"F": 0.0, "T": 0.0, "x": 0.0, "v": 0.0, "w": 0.0, "hist": 0.0}
    flips_total, flips_max, at_bound_total = 0, 0, 0
    for step in range(100):
        seed_oracle_from(oc, sc)
        sc.step(1)
        oc.step(1)
        assert sc.synchronize() == 0
        F, T = sc.forces()
        Fo, To = oc.forces()
        st, so = sc.state(), oc.state()
        e = {"F": rel(F, Fo), "T": rel(T, To),
             "x": float(np.abs(st["x"] - so["x"]).max() / rmin),
             "v": rel(st["v"], so["v"]), "w": rel(st["w"], so["w"])}
        k, h = sc.contacts()
        ko, ho = oc.contacts()
        assert np.array_equal(k, ko), f"{name} step {step}: contact sets differ"
        if len(ho):
            scale = max(np.abs(ho).max(), 1e-300)
            per = np.abs(h - ho).max(axis=1) / scale
            coul = oc.coulomb()
            at_bound = (np.abs(coul - 1.0) <= COULOMB_BAND).any(axis=1)
            at_bound_total += int(at_bound.sum())
            off = per > 1e-4
            assert not (off & ~at_bound).any(), (
                f"{name} step {step}: springs differ away from the Coulomb bound",
                k[off & ~at_bound][:5], per[off & ~at_bound][:5], coul[off & ~at_bound][:5])
            nflip = int((off & at_bound).sum())
            flips_total += nflip
            flips_max = max(flips_max, nflip)
            assert nflip <= MAX_FLIPS_PER_STEP, (name, step, nflip)
            e["hist"] = float(per[~at_bound].max()) if (~at_bound).any() else 0.0
        for key, val in e.items():
            worst[key] = max(worst[key], val)
        bad = {key: val for key, val in e.items()
               if not val <= (1e-5 if key in ("F", "T", "x") else 1e-4)}
        assert not bad, f"{name} step {step}: {bad}; all {e}"
    assert len(ko) > 0, f"{name}: scene has no contacts"
    print(f"{name}/{PREC_NAME[precision]}: worst {worst}; branch flips {flips_total} (max {flips_max} a step) "
          f"among {at_bound_total} contact-steps at the Coulomb bound")


@pytest.mark.parametrize("precision", [0, 1, 2], ids=["fp64", "mixed", "mixed64"])
def test_free_run_from_settled_column(dem, oracle_mod, precision):
    # The column-collapse workload's 2,000-sphere case (log-normal radii on a
    # lattice without initial overlaps, walls 3 column widths out so no sphere
    # rolls off the floor), collapsed and settled on the GPU in the precision
    # under test (150,000 steps, about 1 s), then 100 free steps of the GPU and
    # of the oracle seeded once with the settled state and friction history:
    # forces, torques and positions within the stated tolerance (1e-12 FP64,
    # 1e-5 mixed) after 100 steps, contact sets identical.  At rest a contact
    # that sits at its Coulomb bound can still take the other branch in FP32,
    # but its spring then moves by dt |v| with |v| near zero.
    s = scenes.column_scene(n=2000, seed=3, walls=3.0)
    sc = dem.Scene.from_dict(s, precision=precision, record_forces=True)
    sc.step(150000)
    assert sc.synchronize() == 0
    oc = oracle_scene(oracle_mod, s)
    seed_oracle_from(oc, sc)
    st0 = sc.state()
    vmax = float(np.abs(st0["v"]).max())
    assert vmax < 0.05, vmax  # settled: slow creep at most
    sc.step(100)
    oc.step(100)
    assert sc.synchronize() == 0
    # At rest the torques, velocities and spins are near zero (each particle's
    # contact torques balance), so max|ref| of those arrays is no scale for
    # them; they are measured against the scales the contact forces set over
    # the run: torque R_max max|F|, velocity max|F|/m_min times the run time,
    # spin that velocity over R_min.  Forces (which carry the weight), springs
    # and positions keep the relative measures of the other tests.
    tol = TOL[precision]
    F, T = sc.forces()
    Fo, To = oc.forces()
    st, so = sc.state(), oc.state()
    k, h = sc.contacts()
    ko, ho = oc.contacts()
    assert np.array_equal(k, ko), "contact sets differ"
    R = s["R"]
    rmin, rmax = float(R.min()), float(R.max())
    fmax = float(np.abs(Fo).max())
    mmin = 4.0 / 3.0 * math.pi * s["params"]["rho"] * rmin ** 3
    vscale = fmax / mmin * 100 * s["params"]["dt"]
    errs = {"F": rel(F, Fo), "x": float(np.abs(st["x"] - so["x"]).max() / rmin),
            "hist": rel(h, ho),
            "T": float(np.abs(T - To).max() / (rmax * fmax)),
            "v": float(np.abs(st["v"] - so["v"]).max() / vscale),
            "w": float(np.abs(st["w"] - so["w"]).max() / (vscale / rmin))}
    coul = oc.coulomb()
    print(f"settled column, precision {precision}: max |v| at start {vmax:.3e} m/s, "
          f"max|T| {np.abs(To).max():.3e} of R_max max|F| {rmax * fmax:.3e}, errors {errs}, "
          f"contacts within 1e-4 of the Coulomb bound at the end: "
          f"{int((np.abs(coul - 1.0) <= 1e-4).any(axis=1).sum())} of {len(coul)}")
    bad = {key: val for key, val in errs.items()
           if not val <= (tol if key in ("F", "T", "x") or precision == 0 else 10 * tol)}
    assert not bad, (bad, errs)


def test_parity_ragged_sizes_and_tiny_scenes(dem, oracle_mod):
    # sizes that are not a multiple of the block, down to one particle
    for n in (1, 2, 3, 37, 129):
        s = scenes.box_scene(n=n, seed=10 + n, speed=0.4, size=(0.012, 0.012, 0.02))
        sc, oc = run_pair(dem, oracle_mod, s, 60, 0)
        st, so = sc.state(), oc.state()
        assert np.abs(st["x"] - so["x"]).max() / 0.9e-3 <= 1e-12
        assert rel(st["v"], so["v"]) <= 1e-12


def test_runs_reproduce_bitwise(dem):
    for prec in (0, 1, 2):
        s = scenes.box_scene(n=800, seed=5, speed=0.5)
        outs = []
        for _ in range(2):
            sc = dem.Scene.from_dict(s, precision=prec)
            sc.step(150)
            outs.append(sc.state())
        for key in outs[0]:
            assert np.array_equal(outs[0][key], outs[1][key]), (prec, key)


def test_result_independent_of_skin(dem):
    # sums run in caller-index order over touching contacts only, so the skin
    # (hence the list and the rebuild schedule) cannot change a single bit
    for prec in (0, 1, 2):
        s = scenes.box_scene(n=800, seed=6, speed=0.5)
        st = []
        rebuilds = []
        for skin in (0.05e-3, 0.4e-3):
            sc = dem.Scene.from_dict(s, precision=prec, skin=skin)
            sc.step(200)
            st.append(sc.state())
            rebuilds.append(sc.stats()["rebuilds"])
        assert rebuilds[0] > rebuilds[1]
        for key in st[0]:
            assert np.array_equal(st[0][key], st[1][key]), (prec, key)


def test_save_load_resumes_bitwise(dem):
    for prec in (0, 1, 2):
        s = scenes.drum_scene(n=1500, seed=4, n_theta=32, n_rings=4, nn_dist=2.3e-3,
                              radius=0.022)
        a = dem.Scene.from_dict(s, precision=prec)
        a.step(120)
        blob = a.save()
        a.step(80)
        ref = a.state()
        b = dem.Scene.from_dict(s, precision=prec)
        b.load(blob)
        b.step(80)
        got = b.state()
        for key in ref:
            assert np.array_equal(ref[key], got[key]), (prec, key)


def test_step_chunks_give_the_same_bits(dem):
    # The pose of a rotating mesh is computed one step ahead into a buffer of
    # the step's parity; graphs of 1 and 16 steps, phase-timed steps and a
    # save/load at an odd step must all see the same poses.
    for prec in (0, 1):
        s = scenes.drum_scene(n=1500, seed=4, n_theta=32, n_rings=4, nn_dist=2.3e-3,
                              radius=0.022)
        a = dem.Scene.from_dict(s, precision=prec)
        a.step(77)
        ref = a.state()
        b = dem.Scene.from_dict(s, precision=prec)
        b.step(1)
        b.step_timed(3)
        b.step(17)
        b.step(32)
        blob = b.save()  # at step 53
        b.step_timed(1)
        b.step(23)
        c = dem.Scene.from_dict(s, precision=prec)
        c.load(blob)
        c.step(24)
        for got in (b.state(), c.state()):
            for key in ref:
                assert np.array_equal(ref[key], got[key]), (prec, key)


def test_capacity_overflow_is_reported_not_corrupting(dem):
    s = scenes.lattice_box_scene((6, 6, 6), spacing=1.9e-3)
    sc = dem.Scene.from_dict(s, precision=0, max_neighbors=2)
    sc.step(5)
    assert sc.synchronize() == dem.DEM_ERR_CAPACITY
    # the step that found the overflow did no work: the state is the initial one
    n = sc.n
    x, v, w, q = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 4))
    assert sc.read_state_into(x, v, w, q) == dem.DEM_ERR_CAPACITY
    np.testing.assert_array_equal(x, s["x"])
    np.testing.assert_array_equal(v, s["v"])


def test_pair_sides_give_opposite_forces_bit_for_bit(dem):
    # In the FP32 steps both particles of a pair evaluate it, each with itself
    # as body i of the law; the results must still be exact opposites (and
    # each side's copy of the friction springs must stay consistent).  Sixty
    # isolated pairs with random overlaps, approach speeds, sliding and spins
    # and low friction (so springs go static and kinetic), 150 steps: every
    # step each particle's only contact gives it exactly minus its partner's
    # force, in both FP32 precisions.
    rng = np.random.default_rng(41)
    k = 60
    R = rng.uniform(0.8e-3, 1.2e-3, 2 * k)
    x = np.zeros((2 * k, 3))
    v = rng.normal(0.0, 0.02, (2 * k, 3))
    w = rng.normal(0.0, 20.0, (2 * k, 3))
    for i in range(k):
        n = rng.normal(size=3)
        n /= np.linalg.norm(n)
        x[2 * i] = (0.01 * i, 0.0, 0.0)
        x[2 * i + 1] = x[2 * i] + (R[2 * i] + R[2 * i + 1] - rng.uniform(1e-6, 2e-5)) * n
        v[2 * i + 1] -= 0.02 * n  # approaching
    q = np.zeros((2 * k, 4))
    q[:, 0] = 1.0
    params = scenes.base_params(g=(0.0, 0.0, 0.0), mu_s=0.1, mu_r=0.02, mu_t=0.02,
                                dt=2e-6)
    for prec in (1, 2):
        sc = dem.Scene(params, R, x, v, w, q, precision=prec, record_forces=True)
        touching = 0
        for step in range(150):
            sc.step(1)
            F, _ = sc.forces()
            assert np.array_equal(F[0::2], -F[1::2]), (prec, step)
            touching += int(np.count_nonzero(np.abs(F[0::2]).sum(axis=1)))
        assert touching > 60 * 50, touching


def test_capacity_overflow_regrows_and_retries(dem):
    # A list overflow is found while the lists are rebuilt, before the step
    # does any work; the binding saves the scene, creates it again with twice
    # the capacities, loads the blob and takes the lost steps again.  Results
    # do not depend on the capacities, so the run ends with the bits of a run
    # that never overflowed.
    s = scenes.lattice_box_scene((6, 6, 6), seed=2, spacing=1.9e-3, jitter=2e-5, speed=0.05)
    for prec in (0, 1):
        ref = dem.Scene.from_dict(s, precision=prec)
        ref.step(64)
        want = ref.state()
        sc = dem.Scene.from_dict(s, precision=prec, max_neighbors=2, max_mesh_contacts=1)
        regrows = sc.step_regrowing(64, chunk=16)
        assert regrows >= 2, regrows
        assert sc.synchronize() == 0 and sc.stats()["steps"] == 64
        got = sc.state()
        for key in want:
            assert np.array_equal(want[key], got[key]), (prec, key)


def test_nonfinite_state_is_reported_and_stops_the_run(dem):
    # A NaN planted in one velocity of a saved scene (host side; nothing on
    # the device faults): the next step's integration finds a non-finite state,
    # sets the sticky DEM_ERR_NONFINITE, and later steps do no work.
    import ctypes
    import struct
    for prec in (0, 1):
        s = scenes.box_scene(n=300, seed=12, speed=0.3)
        sc = dem.Scene.from_dict(s, precision=prec)
        sc.step(10)
        assert sc.synchronize() == 0
        blob = bytearray(sc.save())
        n = sc.n
        # header (4 x 8 B), parameters, step / active / draws / carry (4 x 8 B),
        # then the P records (32 B each), then the V records: x of particle 5
        off = 32 + ctypes.sizeof(dem.dem_params) + 32 + n * 32 + 5 * 32
        if prec == 0:
            struct.pack_into("<d", blob, off, float("nan"))
        else:
            struct.pack_into("<f", blob, off, float("nan"))
        sc.load(bytes(blob))
        sc.step(1)
        assert sc.synchronize() == dem.DEM_ERR_NONFINITE
        steps = sc.stats()["steps"]
        x0, v0, w0, q0 = (np.empty((n, k)) for k in (3, 3, 3, 4))
        assert sc.read_state_into(x0, v0, w0, q0) == dem.DEM_ERR_NONFINITE
        sc.step(20)
        assert sc.synchronize() == dem.DEM_ERR_NONFINITE
        assert sc.stats()["steps"] == steps
        x1, v1, w1, q1 = (np.empty((n, k)) for k in (3, 3, 3, 4))
        sc.read_state_into(x1, v1, w1, q1)
        assert np.array_equal(x0, x1, equal_nan=True) and np.array_equal(v0, v1, equal_nan=True)
        assert np.isnan(v0[5, 0])


def test_invalid_inputs_are_rejected(dem):
    s = scenes.box_scene(n=20, seed=1)
    bad = dict(s)
    bad["params"] = dict(s["params"], nu=0.6)  # Table 2: nu in (-1, 0.5]
    with pytest.raises(dem.DemError) as e:
        dem.Scene.from_dict(bad)
    assert e.value.code == dem.DEM_ERR_INVALID
    x = s["x"].copy()
    x[3, 1] = np.nan
    with pytest.raises(dem.DemError):
        dem.Scene(s["params"], s["R"], x)
    R = s["R"].copy()
    R[0] = 0.0
    with pytest.raises(dem.DemError):
        dem.Scene(s["params"], R, s["x"])


def test_momentum_conserved_at_scale(dem):
    # property that holds at any size: no walls, no gravity, friction and
    # damping on -- the total momentum changes only by round-off
    s = scenes.lattice_box_scene((40, 40, 40), seed=8, spacing=1.97e-3, jitter=3e-5,
                                 speed=0.05, spin=20.0, walls=False, gravity=False)
    R = s["R"]
    m = 4 / 3 * math.pi * 2500 * R ** 3
    for prec in (0, 1):
        sc = dem.Scene.from_dict(s, precision=prec)
        p0 = (m[:, None] * s["v"]).sum(0)
        scale = (m[:, None] * np.abs(s["v"])).sum()
        sc.step(200)
        p1 = (m[:, None] * sc.state()["v"]).sum(0)
        tol = 1e-12 if prec == 0 else 2e-6
        assert np.abs(p1 - p0).max() <= tol * scale, prec
        assert sc.stats()["pair_contacts"] > 10000


def test_fp64_one_evaluation_per_pair_is_bitwise_the_two_sided_scheme(dem, monkeypatch):
    # Each pair is evaluated once and its result handed to the partner; the
    # environment switch selects the scheme that evaluates it from both sides.
    # Same values, summed in the same order: in DEM_FP64 (no contraction) the
    # same bits.
    s = SCENES["drum_small"]()
    out = []
    for two in ("0", "1"):
        monkeypatch.setenv("DEM_FP64_TWO_SIDED", two)
        sc = dem.Scene.from_dict(s, precision=0, record_forces=True)
        sc.step(150)
        st = sc.state()
        out.append((st, sc.forces(), sc.contacts(), sc.stats()))
    for key in ("x", "v", "w", "q"):
        assert np.array_equal(out[0][0][key], out[1][0][key]), key
    assert np.array_equal(out[0][1][0], out[1][1][0]) and np.array_equal(out[0][1][1], out[1][1][1])
    assert np.array_equal(out[0][2][0], out[1][2][0]) and np.array_equal(out[0][2][1], out[1][2][1])
    assert out[0][3]["pair_contacts"] == out[1][3]["pair_contacts"] > 0
