"""The allocation-free entry point dem_contact_forces_noalloc.

It serves callers that must not allocate device memory (a real-time loop,
where an allocation can stall, or a host whose device memory belongs to
another allocator).  It evaluates the contact force and torque sums of a
state without friction history, i.e. what the first step of a scene
computes, using a fixed scratch array inside the library.  Checked through
the C ABI against the existing path (dem_scene_create + dem_step(1) +
dem_read_forces, DEM_FP64) at the FP64 tolerance of the other tests, on
several calls in a row so the shared scratch array is reused, and against the
oracle's first step evaluated particle by particle.  Inputs it must refuse
(radius above its bound, a particle outside the box, a crowded cell) are
reported by the device and leave the next call unaffected.  This file is
collected last on purpose.
"""
import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_12610_gb300 import build
    build.build()
    from paper_2507_12610_gb300 import dem
    dem.load()
    return torch, dem


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def reference_first_step(dem, s):
    sc = dem.Scene(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"], precision=dem.DEM_FP64,
                   record_forces=True)
    sc.step(1)
    assert sc.synchronize() == 0
    F, T = sc.forces()
    sc.close()
    return F, T


def noalloc(torch, dem, s, rmax=None, box=None):
    dev = torch.device("cuda")
    n = len(s["R"])
    t = {k: torch.tensor(np.ascontiguousarray(s[k]), dtype=torch.float64, device=dev)
         for k in ("R", "x", "v", "w")}
    F = torch.empty((n, 3), dtype=torch.float64, device=dev)
    T = torch.empty((n, 3), dtype=torch.float64, device=dev)
    rmax = float(s["R"].max()) if rmax is None else rmax
    if box is None:
        lo = s["x"].min(axis=0) - 2 * rmax
        hi = s["x"].max(axis=0) + 2 * rmax
    else:
        lo, hi = box
    torch.cuda.synchronize()
    rc = dem.contact_forces_noalloc(s["params"], n, rmax, t["R"].data_ptr(), t["x"].data_ptr(),
                                    t["v"].data_ptr(), t["w"].data_ptr(), F.data_ptr(),
                                    T.data_ptr(), (lo, hi),
                                    stream=torch.cuda.current_stream().cuda_stream)
    return rc, F.cpu().numpy(), T.cpu().numpy()


def test_noalloc_matches_first_step_on_consecutive_calls(env):
    torch, dem = env
    a = scenes.lattice_box_scene((14, 14, 14), seed=31, spacing=1.95e-3, jitter=3e-5,
                                 speed=0.05, spin=30.0, walls=False)
    b = scenes.lattice_box_scene((10, 12, 9), seed=32, spacing=1.97e-3, jitter=2e-5,
                                 speed=0.1, spin=10.0, walls=False)
    refs = {}
    for name, s in (("a", a), ("b", b), ("a", a)):
        if name not in refs:
            refs[name] = reference_first_step(dem, s)
        F_ref, T_ref = refs[name]
        assert np.abs(F_ref).max() > 0
        rc, F, T = noalloc(torch, dem, s)
        assert rc == dem.DEM_OK, dem.status_string(rc)
        assert rel(F, F_ref) <= TOL, (name, rel(F, F_ref))
        assert rel(T, T_ref) <= TOL, (name, rel(T, T_ref))


def test_noalloc_rejects_sizes_beyond_its_limit(env):
    torch, dem = env
    s = scenes.lattice_box_scene((4, 4, 4), seed=33, walls=False)
    dev = torch.device("cuda")
    buf = torch.zeros(64 * 4, dtype=torch.float64, device=dev)
    p = buf.data_ptr()
    lo, hi = (-0.01, -0.01, 0.0), (0.01, 0.01, 0.02)
    rc = dem.contact_forces_noalloc(s["params"], 131073, 1e-3, p, p, p, p, p, p, (lo, hi))
    assert rc == dem.DEM_ERR_INVALID
    # too many cells for the fixed scratch: a 1 m box with 2 mm cells
    rc = dem.contact_forces_noalloc(s["params"], 64, 1e-3, p, p, p, p, p, p,
                                    ((0, 0, 0), (1.0, 1.0, 1.0)))
    assert rc == dem.DEM_ERR_INVALID


def test_noalloc_matches_the_oracle_first_step(env, oracle_mod):
    # the oracle's first step (no friction history), particle by particle over
    # all partners in ascending index, on a sample of the particles
    torch, dem = env
    s = scenes.lattice_box_scene((12, 12, 12), seed=34, spacing=1.95e-3, jitter=3e-5,
                                 speed=0.05, spin=30.0, walls=False)
    rc, F, T = noalloc(torch, dem, s)
    assert rc == dem.DEM_OK, dem.status_string(rc)
    ids = np.random.default_rng(3).choice(len(s["R"]), 300, replace=False)
    o = oracle_mod.sample_first_step(s["params"], s["R"], s["x"], s["v"], s["w"], s["q"],
                                     None, None, None, ids)
    assert np.abs(o["F"]).max() > 0
    assert rel(F[ids], o["F"]) <= TOL, rel(F[ids], o["F"])
    assert rel(T[ids], o["T"]) <= TOL, rel(T[ids], o["T"])


def test_noalloc_refuses_bad_inputs_on_the_device(env):
    torch, dem = env
    s = scenes.lattice_box_scene((6, 6, 6), seed=35, spacing=1.95e-3, speed=0.05, spin=10.0,
                                 walls=False)
    rmax = float(s["R"].max())
    # a radius above the stated bound
    rc, _, _ = noalloc(torch, dem, s, rmax=0.5 * rmax)
    assert rc == dem.DEM_ERR_INVALID
    # a particle outside the box
    lo = s["x"].min(axis=0) - 2 * rmax
    hi = s["x"].max(axis=0) + 2 * rmax
    bad = dict(s, x=s["x"].copy())
    bad["x"][7] = hi + 0.01
    rc, _, _ = noalloc(torch, dem, bad, box=(lo, hi))
    assert rc == dem.DEM_ERR_INVALID
    # more particles in one cell than the scratch allows
    crowd = dict(s, x=s["x"].copy())
    crowd["x"][:80] = s["x"][0] + np.random.default_rng(1).uniform(-1e-4, 1e-4, (80, 3))
    rc, _, _ = noalloc(torch, dem, crowd)
    assert rc == dem.DEM_ERR_CAPACITY
    # the next call starts from a clear status and gives the reference forces
    F_ref, T_ref = reference_first_step(dem, s)
    rc, F, T = noalloc(torch, dem, s)
    assert rc == dem.DEM_OK
    assert rel(F, F_ref) <= TOL and rel(T, T_ref) <= TOL
