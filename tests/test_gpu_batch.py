"""Batched independent scenes with per-scene friction (GPU) against the oracle."""
import numpy as np
import pytest

from paper_2507_12610_gb300 import batch, scenes

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


def small_batch():
    mus = [(0.25, 0.02, 0.05), (0.75, 0.18, 0.15), (0.5, 0.1, 0.0)]
    # a tight lattice (initial overlaps) and coarse funnels keep the oracle quick
    return batch.combine([batch.hopper_scene(n, 50 + k, mus[k], pitch_factor=1.85, n_theta=16,
                                             n_rings=2) for k, n in enumerate((180, 250, 320))])


def oracle_of(oracle_mod, b):
    V, El, rad = scenes.all_elements(b)
    return oracle_mod.OracleScene(b["params"], b["R"], b["x"], b["v"], b["w"], b["q"], V, El,
                                  rad, material=b["material"], material_mu=b["material_mu"])


@pytest.mark.parametrize("precision", [0, 1], ids=["fp64", "mixed"])
def test_batch_matches_oracle(dem, oracle_mod, precision):
    b = small_batch()
    sc = dem.Scene.from_dict(b, precision=precision, record_forces=True)
    oc = oracle_of(oracle_mod, b)
    sc.step(60)
    oc.step(60)
    assert sc.synchronize() == 0
    k, _ = sc.contacts()
    ko, _ = oc.contacts()
    assert np.array_equal(k, ko) and len(ko) > 200
    tol = 1e-12 if precision == 0 else 1e-5
    F, T = sc.forces()
    Fo, To = oc.forces()
    assert np.abs(F - Fo).max() <= tol * np.abs(Fo).max()
    assert np.abs(T - To).max() <= tol * np.abs(To).max()
    assert np.abs(sc.state()["x"] - oc.state()["x"]).max() <= tol * 0.9e-3
    # no contact joins two scenes
    r = np.searchsorted([a for a, _ in b["ranges"]], k, side="right")
    pairs = k[:, 1] >= 0
    assert np.array_equal(r[pairs, 0], r[pairs, 1])


def test_batched_scene_runs_like_the_scene_alone(dem):
    b = small_batch()
    whole = dem.Scene.from_dict(b, precision=0)
    whole.step(300)
    xs = whole.state()["x"]
    for k, (lo, hi) in enumerate(b["ranges"]):
        one = batch.combine([batch.hopper_scene(hi - lo, 50 + k, tuple(b["material_mu"][k]),
                                                pitch_factor=1.85, n_theta=16, n_rings=2)])
        sc = dem.Scene.from_dict(one, precision=0)
        sc.step(300)
        d = xs[lo:hi] - b["offsets"][k] - (sc.state()["x"] - one["offsets"][0])
        assert np.abs(d).max() < 1e-12, k


def test_block_shape_does_not_change_results(dem):
    b = small_batch()
    out = []
    for bw in (4, 8):
        sc = dem.Scene.from_dict(b, precision=1, step_warps=bw)
        sc.step(200)
        out.append(sc.state())
    for key in out[0]:
        assert np.array_equal(out[0][key], out[1][key]), key


def test_hoppers_discharge_at_different_rates(dem):
    b = small_batch()
    sc = dem.Scene.from_dict(b, precision=1)
    sc.step(6000)
    f = batch.discharged(b, sc.state()["x"])
    assert np.all(f > 0.05), f
    best, table = batch.autotune(b, steps=50, warmup=10, dem=dem)
    assert best in table and len(table) == 8
