"""Host side of the batched ensemble: scene packing and combination (no GPU)."""
import numpy as np

from paper_2507_12610_gb300 import batch


def boxes_of(scenes_, off):
    return [(np.asarray(s["box"][0]) + o, np.asarray(s["box"][1]) + o) for s, o in zip(scenes_, off)]


def test_pack_keeps_boxes_apart_by_the_gap():
    rng = np.random.default_rng(3)
    boxes = []
    for _ in range(60):
        lo = rng.uniform(-1, 1, 3)
        boxes.append((lo, lo + rng.uniform(0.01, 0.2, 3)))
    off = batch.pack(boxes, gap=0.01)
    placed = [(np.asarray(lo) + o, np.asarray(hi) + o) for (lo, hi), o in zip(boxes, off)]
    for i in range(len(placed)):
        for j in range(i + 1, len(placed)):
            (a0, a1), (b0, b1) = placed[i], placed[j]
            # separated along at least one axis by the gap
            sep = np.maximum(b0 - a1, a0 - b1)
            assert sep.max() >= 0.01 - 1e-12, (i, j)


def test_combine_concatenates_scenes_with_their_materials():
    sc = [batch.hopper_scene(600, 1, mu=(0.3, 0.1, 0.05), pitch_factor=1.85, n_theta=16,
                             n_rings=2),
          batch.hopper_scene(900, 2, mu=(0.7, 0.0, 0.2), pitch_factor=1.85, n_theta=16,
                             n_rings=2)]
    b = batch.combine(sc)
    n0, n1 = len(sc[0]["R"]), len(sc[1]["R"])
    assert b["ranges"] == [(0, n0), (n0, n0 + n1)]
    assert np.array_equal(b["material"], np.repeat([0, 1], [n0, n1]))
    np.testing.assert_array_equal(b["material_mu"], [sc[0]["mu"], sc[1]["mu"]])
    # each scene moved rigidly by its offset: particles and mesh alike
    for k, (a, e) in enumerate(b["ranges"]):
        np.testing.assert_array_equal(b["x"][a:e], sc[k]["x"] + b["offsets"][k])
    nv0 = sc[0]["verts"].shape[0]
    np.testing.assert_array_equal(b["verts"][:nv0], sc[0]["verts"] + b["offsets"][0])
    assert b["tris"].min() >= 0 and b["tris"][len(sc[0]["tris"]):].min() >= nv0
    # no contact can join two scenes: their packed boxes are apart by the gap
    (a0, a1), (b0, b1) = boxes_of(sc, b["offsets"])
    assert np.maximum(b0 - a1, a0 - b1).max() >= batch.GAP - 1e-12
    # every particle lies in its own scene's packed box
    for k, (a, e) in enumerate(b["ranges"]):
        lo, hi = boxes_of(sc, b["offsets"])[k]
        assert np.all(b["x"][a:e] >= lo) and np.all(b["x"][a:e] <= hi)


def test_discharged_fraction_counts_particles_below_each_outlet():
    sc = [batch.hopper_scene(600, 1, pitch_factor=1.85, n_theta=16, n_rings=2)]
    b = batch.combine(sc)
    x = b["x"].copy()
    assert batch.discharged(b, x)[0] == 0.0
    x[:150, 2] = b["offsets"][0, 2] + b["z_outlet"][0] - 1e-3
    assert batch.discharged(b, x)[0] == 150 / 600
