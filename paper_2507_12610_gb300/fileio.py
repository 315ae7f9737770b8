"""Mesh and particle files (Sec. 6, usage): OFF meshes and CSV frames.

* Mesh: GeomView's Object File Format (OFF).  Each face line lists its vertex
  count (1 point, 2 segment, 3 triangle, 4 rectangle -- the element kinds of
  Sec. 3.3), its vertex indices and, optionally, one integer: the index of the
  face's radius in the list of mesh radii R_mesh (Table 2).  Without it the
  face takes R_mesh[0], the default mesh radius.
* Particles: one CSV table per frame, a header line with the column names and
  one row per particle (radius, position, velocity, angular velocity and
  orientation quaternion).  A run writes 1 + N_frames tables, the initial state
  and one after every N_steps steps; existing files are overwritten.

Numbers are written with 17 significant digits, so a written file reads back
bitwise.  Host-side file handling only: nothing here is on the time-step path.
"""
from __future__ import annotations

import os

import numpy as np

CSV_COLUMNS = ("R", "x", "y", "z", "vx", "vy", "vz", "wx", "wy", "wz", "q0", "q1", "q2", "q3")


def _tokens(path):
    """Whitespace tokens of an OFF file, one list per non-empty line, with
    '#' comments removed."""
    with open(path) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                yield line.split()


def _is_int(tok: str) -> bool:
    try:
        int(tok)
        return True
    except ValueError:
        return False


def read_off(path, radii=(0.0,)):
    """Read an OFF mesh.

    Returns (verts [nv, 3] float64, elems [m, 4] int32 padded with -1,
    elem_radius [m] float64): the radius of face k is radii[index_k], index_k
    the optional integer after its vertex indices (0 if absent).  Faces of more
    than four vertices, indices out of range and radius indices outside
    `radii` raise ValueError.  Colour values that are not a single integer are
    ignored (the face takes radii[0]).
    """
    radii = np.asarray(radii, dtype=np.float64).reshape(-1)
    if radii.size == 0:
        raise ValueError("need at least one mesh radius")
    lines = _tokens(path)
    head = next(lines, None)
    if head is None or not head[0].endswith("OFF"):
        raise ValueError(f"{path}: not an OFF file")
    counts = head[1:] if len(head) > 1 else next(lines)
    nv, nf = int(counts[0]), int(counts[1])
    verts = np.empty((nv, 3))
    for k in range(nv):
        t = next(lines)
        verts[k] = [float(t[0]), float(t[1]), float(t[2])]
    elems = np.full((nf, 4), -1, dtype=np.int32)
    rad = np.empty(nf)
    for k in range(nf):
        t = next(lines)
        m = int(t[0])
        if not 1 <= m <= 4:
            raise ValueError(f"{path}: face {k} has {m} vertices (1 to 4 supported)")
        idx = [int(s) for s in t[1:1 + m]]
        if len(idx) != m or min(idx) < 0 or max(idx) >= nv:
            raise ValueError(f"{path}: face {k} has bad vertex indices")
        elems[k, :m] = idx
        extra = t[1 + m:]
        ri = int(extra[0]) if len(extra) == 1 and _is_int(extra[0]) else 0
        if not 0 <= ri < radii.size:
            raise ValueError(f"{path}: face {k} radius index {ri} outside R_mesh")
        rad[k] = radii[ri]
    return verts, elems, rad


def write_off(path, verts, elems, radius_index=None):
    """Write an OFF mesh; elems rows hold 1-4 vertex indices padded with -1
    (or are (m, 3) triangles); radius_index[k], if given, is appended to face k."""
    verts = np.asarray(verts, dtype=np.float64).reshape(-1, 3)
    el = np.asarray(elems, dtype=np.int64)
    el = el.reshape(-1, el.shape[-1] if el.ndim > 1 else 3)
    with open(path, "w") as f:
        f.write("OFF\n")
        f.write(f"{verts.shape[0]} {el.shape[0]} 0\n")
        for v in verts:
            f.write(" ".join(repr(float(c)) for c in v) + "\n")
        for k, row in enumerate(el):
            ids = [int(i) for i in row if i >= 0]
            line = f"{len(ids)} " + " ".join(str(i) for i in ids)
            if radius_index is not None:
                line += f" {int(radius_index[k])}"
            f.write(line + "\n")


def write_csv(path, R, x, v=None, w=None, q=None):
    """Write one particle table (columns CSV_COLUMNS); missing v, w are zero
    and a missing q is the identity."""
    R = np.asarray(R, dtype=np.float64).reshape(-1)
    n = R.shape[0]
    cols = [R[:, None], np.asarray(x, dtype=np.float64).reshape(n, 3),
            np.zeros((n, 3)) if v is None else np.asarray(v, dtype=np.float64).reshape(n, 3),
            np.zeros((n, 3)) if w is None else np.asarray(w, dtype=np.float64).reshape(n, 3)]
    if q is None:
        q = np.zeros((n, 4))
        q[:, 0] = 1.0
    cols.append(np.asarray(q, dtype=np.float64).reshape(n, 4))
    table = np.hstack(cols)
    tmp = f"{path}.tmp{os.getpid()}"
    with open(tmp, "w") as f:
        f.write(",".join(CSV_COLUMNS) + "\n")
        np.savetxt(f, table, delimiter=",", fmt="%.17g")
    os.replace(tmp, path)


def read_csv(path) -> dict:
    """Read a particle table written by write_csv (or any CSV whose header
    names at least R, x, y, z; absent velocity columns read as zero, absent
    quaternion columns as the identity).  Returns dict R, x, v, w, q."""
    with open(path) as f:
        header = [h.strip() for h in f.readline().strip().split(",")]
    if not {"R", "x", "y", "z"} <= set(header):
        raise ValueError(f"{path}: header must name R, x, y and z")
    data = np.loadtxt(path, delimiter=",", skiprows=1, ndmin=2)
    if data.size == 0:
        data = np.zeros((0, len(header)))
    col = {h: data[:, k] for k, h in enumerate(header)}
    n = data.shape[0]

    def grab(names, default):
        if all(c in col for c in names):
            return np.stack([col[c] for c in names], axis=1)
        out = np.zeros((n, len(names)))
        out[:, 0] = default
        return out

    return {"R": col["R"].copy(), "x": grab(("x", "y", "z"), 0.0),
            "v": grab(("vx", "vy", "vz"), 0.0), "w": grab(("wx", "wy", "wz"), 0.0),
            "q": grab(("q0", "q1", "q2", "q3"), 1.0)}


def frame_path(out_dir, k: int) -> str:
    return os.path.join(out_dir, f"frame_{k:05d}.csv")


def write_frames(scene, out_dir, n_frames: int, n_steps: int):
    """Advance `scene` n_frames x n_steps steps and write 1 + n_frames particle
    tables (the initial state, then one per n_steps steps) into out_dir.

    `scene` needs `R` (radii), `state()` (x, v, w, q) and `step(k)`, as
    `dem.Scene` has.  Returns the list of written paths."""
    os.makedirs(out_dir, exist_ok=True)
    paths = []
    for k in range(n_frames + 1):
        if k:
            scene.step(n_steps)
        st = scene.state()
        p = frame_path(out_dir, k)
        write_csv(p, scene.R, st["x"], st["v"], st["w"], st["q"])
        paths.append(p)
    return paths


def scene_inputs(params: dict, off_path=None, csv_path=None, radii=(0.0,)) -> dict:
    """Scene dictionary (as `dem.Scene.from_dict` takes) from an OFF mesh and a
    particle CSV; mesh faces become elements in file order."""
    if csv_path is None:
        raise ValueError("a particle CSV is needed (spawning is not provided)")
    p = read_csv(csv_path)
    s = dict(params=params, R=p["R"], x=p["x"], v=p["v"], w=p["w"], q=p["q"], verts=None,
             tris=None, tri_radius=None, elems=None, elem_radius=None)
    if off_path is not None:
        V, El, rad = read_off(off_path, radii)
        s.update(verts=V, elems=El, elem_radius=rad)
    return s
