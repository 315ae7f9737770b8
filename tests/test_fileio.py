"""OFF meshes and CSV particle frames (Sec. 6, usage), on the CPU."""
import os

import numpy as np
import pytest

from paper_2507_12610_gb300 import fileio, scenes

OFF_TEXT = """OFF
# a floor plate, a ramp triangle, a bar and a post top
7 4 0
0 0 0
1 0 0
1 1 0
0 1 0
0.5 0.5 1   # apex
0.2 0.8 0.3
0.9 0.8 0.3
4 0 1 2 3
3 0 1 4 2
2 5 6 1
1 4 0.1 0.2 0.3
"""


def test_off_faces_and_radius_indices(tmp_path):
    p = tmp_path / "m.off"
    p.write_text(OFF_TEXT)
    V, El, rad = fileio.read_off(str(p), radii=(0.002, 0.02, 0.01))
    assert V.shape == (7, 3) and V[4].tolist() == [0.5, 0.5, 1.0]
    assert El.tolist() == [[0, 1, 2, 3], [0, 1, 4, -1], [5, 6, -1, -1], [4, -1, -1, -1]]
    # faces 1 and 2 name radius indices 2 and 1; a face without an index, or
    # with a colour that is not one integer, takes R_mesh[0]
    assert rad.tolist() == [0.002, 0.01, 0.02, 0.002]


@pytest.mark.parametrize("bad", ["5 0 1 2 3 4", "3 0 1 9", "3 0 1 2 7"])
def test_off_rejects_bad_faces(tmp_path, bad):
    p = tmp_path / "bad.off"
    p.write_text(f"OFF\n5 1 0\n0 0 0\n1 0 0\n0 1 0\n0 0 1\n1 1 1\n{bad}\n")
    with pytest.raises(ValueError):
        fileio.read_off(str(p), radii=(0.0, 1.0))


def test_off_round_trip_is_bitwise(tmp_path):
    s = scenes.primitives_scene(n_side=(2, 2, 2))
    V, El, rad = scenes.all_elements(s)
    table, index = np.unique(rad, return_inverse=True)
    p = str(tmp_path / "prims.off")
    fileio.write_off(p, V, El, index)
    V2, El2, rad2 = fileio.read_off(p, table)
    assert np.array_equal(V, V2) and np.array_equal(El, El2) and np.array_equal(rad, rad2)


def test_csv_round_trip_is_bitwise(tmp_path):
    rng = np.random.default_rng(0)
    n = 257
    R = rng.uniform(0.8e-3, 1.2e-3, n)
    x, v, w = rng.normal(size=(n, 3)), rng.normal(size=(n, 3)), rng.normal(size=(n, 3)) * 1e3
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    p = str(tmp_path / "p.csv")
    fileio.write_csv(p, R, x, v, w, q)
    assert open(p).readline().strip() == ",".join(fileio.CSV_COLUMNS)
    d = fileio.read_csv(p)
    for k, a in (("R", R), ("x", x), ("v", v), ("w", w), ("q", q)):
        assert np.array_equal(d[k], a), k


def test_csv_other_column_order_and_defaults(tmp_path):
    p = tmp_path / "few.csv"
    p.write_text("z,R,y,x\n3,0.5,2,1\n6,0.25,5,4\n")
    d = fileio.read_csv(str(p))
    assert d["R"].tolist() == [0.5, 0.25]
    assert d["x"].tolist() == [[1, 2, 3], [4, 5, 6]]
    assert not d["v"].any() and not d["w"].any()
    assert d["q"].tolist() == [[1, 0, 0, 0], [1, 0, 0, 0]]
    bad = tmp_path / "bad.csv"
    bad.write_text("x,y,z\n1,2,3\n")
    with pytest.raises(ValueError):
        fileio.read_csv(str(bad))


class _FakeScene:
    """Stands in for dem.Scene: x moves by the number of steps taken."""

    def __init__(self, n):
        self.R = np.full(n, 1e-3)
        self.t = 0

    def step(self, k):
        self.t += k

    def state(self):
        n = self.R.shape[0]
        q = np.zeros((n, 4))
        q[:, 0] = 1
        return {"x": np.full((n, 3), float(self.t)), "v": np.zeros((n, 3)),
                "w": np.zeros((n, 3)), "q": q}


def test_frames_are_initial_state_plus_one_per_interval(tmp_path):
    out = str(tmp_path / "out")
    paths = fileio.write_frames(_FakeScene(5), out, n_frames=3, n_steps=7)
    assert [os.path.basename(p) for p in paths] == [f"frame_{k:05d}.csv" for k in range(4)]
    for k, p in enumerate(paths):
        assert np.all(fileio.read_csv(p)["x"] == 7 * k)
    # a second run overwrites without asking
    paths = fileio.write_frames(_FakeScene(2), out, n_frames=1, n_steps=1)
    assert fileio.read_csv(paths[0])["R"].shape == (2,)


def test_scene_inputs_from_files(tmp_path):
    s = scenes.primitives_scene(n_side=(3, 3, 3))
    V, El, rad = scenes.all_elements(s)
    table, index = np.unique(rad, return_inverse=True)
    fileio.write_off(str(tmp_path / "m.off"), V, El, index)
    fileio.write_csv(str(tmp_path / "p.csv"), s["R"], s["x"], s["v"], s["w"], s["q"])
    d = fileio.scene_inputs(s["params"], str(tmp_path / "m.off"), str(tmp_path / "p.csv"), table)
    assert np.array_equal(d["elems"], El) and np.array_equal(d["elem_radius"], rad)
    assert np.array_equal(d["x"], s["x"]) and np.array_equal(d["q"], s["q"])
