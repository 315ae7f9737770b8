"""Particle spawning (Sec. 3.1) on the GPU against the oracle."""
import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes

pytestmark = pytest.mark.gpu


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


def spawn_scene(n_init=40, n_max=500, attempts=40, every=10, seed=21, spin=0.0):
    """A floor plate (radius 0.2 mm), a few resting spheres, and a spawn box
    above them: spawned spheres fall onto the floor and each other.  spin:
    the plate turns about the vertical axis at this rate (rad/s)."""
    rng = np.random.default_rng(seed)
    V = np.array([[-0.015, -0.015, 0], [0.015, -0.015, 0], [0.015, 0.015, 0],
                  [-0.015, 0.015, 0]], dtype=np.float64)
    E = np.array([[0, 1, 2, 3]], dtype=np.int32)
    g = np.stack(np.meshgrid(np.arange(8), np.arange(5), indexing="ij"), -1).reshape(-1, 2)
    x = np.zeros((n_init, 3))
    x[:, :2] = (g[:n_init] - [3.5, 2]) * 2.3e-3
    R = rng.uniform(0.9e-3, 1.1e-3, n_init)
    x[:, 2] = R + 0.2e-3 - 2e-6  # pressed slightly into the floor
    sp = dict(n_max=n_max, lo=(-0.009, -0.009, 0.0035), hi=(0.009, 0.009, 0.007),
              r_min=0.9e-3, r_max=1.1e-3, v0=(0.0, 0.0, -1.0), w0=(0.0, 0.0, 5.0),
              attempts=attempts, every=every, seed=seed)
    p = scenes.base_params(mesh_omega=(0.0, 0.0, spin), mesh_center=(0.0, 0.0, 0.0))
    return dict(params=p, R=R, x=x, v=None, w=None, q=None, verts=V, tris=None,
                tri_radius=None, elems=E, elem_radius=np.array([0.2e-3]), spawn=sp)


def oracle_of(oracle_mod, s):
    V, El, rad = scenes.all_elements(s)
    return oracle_mod.OracleScene(s["params"], s["R"], s["x"], verts=V, tris=El,
                                  tri_radius=rad, spawn=s["spawn"])


@pytest.mark.parametrize("spin", [0.0, 20.0], ids=["still", "turning"])
@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_spawning_matches_oracle(dem, oracle_mod, precision, spin):
    # turning: the floor plate spins in its plane, so its element list is
    # looked up in the plate's frame by the list build and by the spawn test
    s = spawn_scene(spin=spin)
    sc = dem.Scene.from_dict(s, precision=precision, record_forces=True)
    oc = oracle_of(oracle_mod, s)
    # DEM_MIXED: 300 steps, the impacts of spawned spheres at 1 m/s amplify
    # its 1e-7 differences further on; DEM_FP64 stays at ~1e-13 for 600
    steps = 600 if precision == 0 else 300
    sc.step(steps)
    oc.step(steps)
    assert sc.synchronize() == 0
    st = sc.stats()
    assert st["active"] == oc.active and st["capacity"] == oc.n == 500
    assert oc.active > 150
    # radii come from the same uniforms by the same formula: identical (to the
    # 48 bits of the two floats DEM_MIXED keeps)
    if precision == 0:
        assert np.array_equal(sc.radii(), oc.radii())
    else:
        assert np.allclose(sc.radii(), oc.radii(), rtol=1e-14, atol=0)
    k, h = sc.contacts()
    ko, ho = oc.contacts()
    assert np.array_equal(k, ko) and len(ko) > 50
    tol = 1e-12 if precision == 0 else 1e-5
    F, T = sc.forces()
    Fo, To = oc.forces()
    assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max()
    assert np.abs(T - To).max() <= tol * np.abs(To).max()
    a, b = sc.state(), oc.state()
    assert np.abs(a["x"] - b["x"]).max() <= tol * 0.9e-3
    # rows awaiting spawning read as zeros
    n = oc.active
    assert not a["x"][n:].any() and np.all(sc.radii()[n:] == 0)


def test_spawning_from_no_particles_and_resume(dem, oracle_mod):
    s = spawn_scene(n_init=0, n_max=120, attempts=8, every=3, seed=4)
    s["R"], s["x"] = np.zeros(0), np.zeros((0, 3))
    a = dem.Scene.from_dict(s, precision=0)
    a.step(90)
    blob = a.save()
    a.step(90)
    b = dem.Scene.from_dict(s, precision=0)
    b.load(blob)
    b.step(90)
    assert a.active == b.active > 50
    for key in ("x", "v", "w", "q"):
        assert np.array_equal(a.state()[key], b.state()[key]), key
    oc = oracle_of(oracle_mod, s)
    oc.step(180)
    assert oc.active == a.active and np.array_equal(a.radii(), oc.radii())
