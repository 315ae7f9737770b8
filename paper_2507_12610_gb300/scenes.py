"""Seeded synthetic scenes (particles, meshes, material parameters).

This module only generates inputs: radii, positions, velocities, orientations,
triangle meshes and parameter dictionaries.  It holds none of the contact or
integration arithmetic, so both the CUDA path and its checks may use it.

Material defaults follow Table 2 of arXiv 2507.12610 (E = 1 MPa, nu = 0.3,
eta = 0); density, friction, restitution and geometry follow the workloads
below.  The time steps are 1/50 of the elastic Hertz contact time of two
R_min spheres whose peak indentation is 10 % of 2R* (the collision that Eq. dt
is stated to resolve with about a dozen steps, Sec. 2.3); the numbers are
written out here and checked against the closed form by the test suite.

Workloads:
  box     1,000 spheres, R ~ U[0.9, 1.1] mm, rho 2500, mu 0.5/0.1/0.1, e_n 0.5,
          random sequential (non-overlapping) start in a 20 x 20 x 60 mm box of
          12 triangles, gravity 9.81.
  column  log-normal radii (median 1 mm, sigma 0.2, truncated at +-3 sigma),
          square column of aspect ratio 2 on a floor mesh, same friction set.
  drum    R ~ U[0.8, 1.2] mm, closed cylinder of 4,096 triangles (128 facets
          around, 15 rings along the axis, fan caps) turning at 30 rpm about the
          horizontal x axis, mu 0.4/0.05/0.05, 35 % fill at packing ~0.6.
"""
from __future__ import annotations

import math

import numpy as np

# dt = t_c / 50 (see module docstring); t_c for R_min = 0.9, 0.5488, 0.8 mm.
DT_BOX = 1.0589647798775054e-05
DT_COLUMN = 6.457468815672489e-06
DT_DRUM = 9.413020265577825e-06

RPM_30 = 30.0 * 2.0 * math.pi / 60.0


def base_params(**over) -> dict:
    p = dict(E=1.0e6, nu=0.3, rho=2500.0, e_n=0.5, mu_s=0.5, mu_r=0.1, mu_t=0.1, eta=0.0,
             g=(0.0, 0.0, -9.81), dt=DT_BOX, mesh_omega=(0.0, 0.0, 0.0),
             mesh_center=(0.0, 0.0, 0.0))
    p.update(over)
    return p


def _unit_quaternions(rng, n):
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q


def box_mesh(lo, hi):
    """Axis-aligned closed box as 12 triangles (two per face)."""
    x0, y0, z0 = lo
    x1, y1, z1 = hi
    V = np.array([[x0, y0, z0], [x1, y0, z0], [x1, y1, z0], [x0, y1, z0],
                  [x0, y0, z1], [x1, y0, z1], [x1, y1, z1], [x0, y1, z1]], dtype=np.float64)
    faces = [(0, 1, 2, 3), (4, 7, 6, 5), (0, 4, 5, 1), (1, 5, 6, 2), (2, 6, 7, 3), (3, 7, 4, 0)]
    T = []
    for a, b, c, d in faces:
        T.append((a, b, c))
        T.append((a, c, d))
    return V, np.array(T, dtype=np.int32)


def drum_mesh(radius, length, n_theta=128, n_rings=15):
    """Closed cylinder about the x axis centred at the origin.

    Side: n_rings x n_theta quads split in two triangles; caps: triangle fans.
    4,096 triangles for n_theta = 128, n_rings = 15.
    """
    th = 2.0 * math.pi * np.arange(n_theta) / n_theta
    xs = -0.5 * length + length * np.arange(n_rings + 1) / n_rings
    ring = np.stack([np.cos(th) * radius, np.sin(th) * radius], axis=1)
    V = [np.array([x, y, z]) for x in xs for (y, z) in ring]
    c0 = len(V)
    V.append(np.array([-0.5 * length, 0.0, 0.0]))
    c1 = len(V)
    V.append(np.array([0.5 * length, 0.0, 0.0]))
    T = []
    for iz in range(n_rings):
        for it in range(n_theta):
            a = iz * n_theta + it
            b = iz * n_theta + (it + 1) % n_theta
            c = (iz + 1) * n_theta + it
            d = (iz + 1) * n_theta + (it + 1) % n_theta
            T.append((a, c, d))
            T.append((a, d, b))
    last = n_rings * n_theta
    for it in range(n_theta):
        T.append((c0, (it + 1) % n_theta, it))
        T.append((c1, last + it, last + (it + 1) % n_theta))
    return np.array(V, dtype=np.float64), np.array(T, dtype=np.int32)


def _scene(name, seed, params, R, x, v, w, q, V, T, tri_radius, domain, elems=None,
           elem_radius=None):
    return dict(name=name, seed=seed, params=params, R=R, x=x, v=v, w=w, q=q, verts=V,
                tris=T, tri_radius=tri_radius, elems=elems, elem_radius=elem_radius,
                domain=domain)


def all_elements(s):
    """(verts, elements (m, 4) padded with -1, radii) of a scene's mesh: its
    triangles first, then its other elements, the numbering of contact keys."""
    T = np.asarray(s["tris"] if s.get("tris") is not None else np.zeros((0, 3)), dtype=np.int32)
    El = np.full((T.shape[0], 4), -1, dtype=np.int32)
    El[:, :3] = T.reshape(-1, 3)
    rt = s.get("tri_radius")
    rad = np.zeros(T.shape[0]) if rt is None else np.asarray(rt, dtype=np.float64)
    if s.get("elems") is not None and len(s["elems"]):
        El = np.vstack([El, np.asarray(s["elems"], dtype=np.int32).reshape(-1, 4)])
        er = s.get("elem_radius")
        rad = np.concatenate([rad, np.zeros(len(s["elems"])) if er is None
                              else np.asarray(er, dtype=np.float64)])
    return np.asarray(s["verts"], dtype=np.float64).reshape(-1, 3), El, rad


def box_scene(n=1000, seed=1, speed=0.0, gravity=True, size=(0.020, 0.020, 0.060),
              r_range=(0.9e-3, 1.1e-3), **over):
    """Random sequential non-overlapping start in an axis-aligned box."""
    rng = np.random.default_rng(seed)
    lx, ly, lz = size
    lo = np.array([-lx / 2, -ly / 2, 0.0])
    hi = np.array([lx / 2, ly / 2, lz])
    R = rng.uniform(r_range[0], r_range[1], size=n)
    X = np.empty((n, 3))
    placed = 0
    attempts = 0
    while placed < n:
        attempts += 1
        if attempts > 200000 * max(1, n // 1000):
            raise RuntimeError("random sequential placement did not converge")
        r = R[placed]
        p = rng.uniform(lo + r, hi - r)
        if placed:
            d = np.linalg.norm(X[:placed] - p, axis=1)
            if np.any(d < R[:placed] + r):
                continue
        X[placed] = p
        placed += 1
    v = rng.normal(scale=speed, size=(n, 3)) if speed > 0 else np.zeros((n, 3))
    w = np.zeros((n, 3))
    q = _unit_quaternions(rng, n)
    V, T = box_mesh(lo, hi)
    params = base_params(dt=DT_BOX, g=(0.0, 0.0, -9.81 if gravity else 0.0))
    params.update(over)
    return _scene("box", seed, params, R, X, v, w, q, V, T, np.zeros(len(T)), (lo, hi))


def lattice_box_scene(n_side=(10, 10, 10), seed=2, spacing=2.0e-3, r_range=(0.9e-3, 1.1e-3),
                      jitter=0.0, speed=0.0, spin=0.0, walls=True, gravity=True, **over):
    """Simple cubic lattice in a box; spacing below 2R gives initial overlaps."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = n_side
    gi = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                  axis=-1).reshape(-1, 3).astype(np.float64)
    n = gi.shape[0]
    R = rng.uniform(r_range[0], r_range[1], size=n)
    X = (gi - 0.5 * (np.array([nx, ny, 0]) - 1)) * spacing
    X[:, 2] += r_range[1]
    if jitter > 0:
        X += rng.uniform(-jitter, jitter, size=X.shape)
    v = rng.normal(scale=speed, size=(n, 3)) if speed > 0 else np.zeros((n, 3))
    w = rng.normal(scale=spin, size=(n, 3)) if spin > 0 else np.zeros((n, 3))
    q = _unit_quaternions(rng, n)
    lo = X.min(axis=0) - r_range[1] * 1.01
    hi = X.max(axis=0) + r_range[1] * 1.01
    lo[2] = 0.0
    if walls:
        V, T = box_mesh(lo, hi)
    else:
        V, T = np.zeros((0, 3)), np.zeros((0, 3), dtype=np.int32)
    params = base_params(dt=DT_BOX, g=(0.0, 0.0, -9.81 if gravity else 0.0))
    params.update(over)
    return _scene("lattice_box", seed, params, R, X, v, w, q, V, T, np.zeros(len(T)), (lo, hi))


def column_scene(n=2000, seed=3, median=1.0e-3, sigma=0.2, gap=0.05e-3, spacing=None,
                 walls=None, **over):
    """Square column of aspect ratio 2 (height = 2 x width) on a floor mesh.

    Particles sit on a jittered cubic lattice of pitch `spacing` (default
    2 R_max + gap: no overlaps); a smaller pitch gives initial contacts.
    `walls` (optional) closes the floor with four vertical walls at +-walls
    column widths from the axis, so no particle can leave it.
    """
    rng = np.random.default_rng(seed)
    rmin, rmax = median * math.exp(-3 * sigma), median * math.exp(3 * sigma)
    R = np.empty(0)
    while R.size < n:  # truncated log-normal by rejection
        s = np.exp(rng.normal(math.log(median), sigma, size=2 * n))
        R = np.concatenate([R, s[(s >= rmin) & (s <= rmax)]])
    R = R[:n]
    d = 2 * rmax + gap if spacing is None else spacing
    k = 1
    while 2 * k ** 3 < n:
        k += 1
    gi = np.stack(np.meshgrid(np.arange(k), np.arange(k), np.arange(2 * k), indexing="ij"),
                  axis=-1).reshape(-1, 3).astype(np.float64)
    order = np.lexsort((gi[:, 0], gi[:, 1], gi[:, 2]))  # fill bottom layers first
    gi = gi[order][:n]
    X = np.empty((n, 3))
    X[:, 0] = (gi[:, 0] - 0.5 * (k - 1)) * d
    X[:, 1] = (gi[:, 1] - 0.5 * (k - 1)) * d
    X[:, 2] = 0.5 * d + gi[:, 2] * d
    slack = np.maximum(0.5 * (d - 2 * R), 0.0)[:, None]
    X += rng.uniform(-1.0, 1.0, size=X.shape) * slack * 0.5
    w_col = k * d
    L = 6.0 * w_col
    V = np.array([[-L, -L, 0.0], [L, -L, 0.0], [L, L, 0.0], [-L, L, 0.0]])
    T = np.array([[0, 1, 2], [0, 2, 3]], dtype=np.int32)
    if walls is not None:
        W, H = walls * w_col, 2.5 * k * d
        V = np.vstack([V, [[-W, -W, 0.0], [W, -W, 0.0], [W, W, 0.0], [-W, W, 0.0],
                           [-W, -W, H], [W, -W, H], [W, W, H], [-W, W, H]]])
        T = np.vstack([T, np.array([[4, 5, 9], [4, 9, 8], [5, 6, 10], [5, 10, 9],
                                    [6, 7, 11], [6, 11, 10], [7, 4, 8], [7, 8, 11]])])
    v = np.zeros((n, 3))
    w = np.zeros((n, 3))
    q = _unit_quaternions(rng, n)
    params = base_params(dt=DT_COLUMN)
    params.update(over)
    lo = np.array([-L, -L, 0.0])
    hi = np.array([L, L, 2 * k * d + 2 * rmax])
    return _scene("column", seed, params, R, X, v, w, q, V, T, np.zeros(len(T)), (lo, hi))


def drum_geometry(n_particles, r_range=(0.8e-3, 1.2e-3), fill=0.35, packing=0.6):
    """Drum radius for the requested fill (length = 2 radius)."""
    r0, r1 = r_range
    mean_r3 = (r1 ** 4 - r0 ** 4) / (4.0 * (r1 - r0))
    solid = n_particles * 4.0 / 3.0 * math.pi * mean_r3
    vol = solid / packing / fill
    radius = (vol / (2.0 * math.pi)) ** (1.0 / 3.0)
    return radius, 2.0 * radius


def fcc_points(lo, hi, a):
    """Face-centred cubic lattice points (lattice constant a) inside [lo, hi]."""
    base = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    n = np.floor((np.asarray(hi) - np.asarray(lo)) / a).astype(int) + 1
    g = np.stack(np.meshgrid(np.arange(n[0]), np.arange(n[1]), np.arange(n[2]), indexing="ij"),
                 axis=-1).reshape(-1, 1, 3)
    P = (g + base[None]).reshape(-1, 3) * a + np.asarray(lo)
    keep = np.all((P >= lo) & (P <= hi), axis=1)
    return P[keep]


def drum_scene(n=1_000_000, seed=5, n_theta=128, n_rings=15, r_range=(0.8e-3, 1.2e-3),
               fill=0.35, rpm=30.0, nn_dist=None, speed=0.01, radius=None, **over):
    """Particles on an FCC lattice in the lower part of a rotating drum.

    nn_dist is the lattice nearest-neighbour distance (default 2 R_max plus a
    small gap, i.e. no overlaps); a smaller value gives initial overlaps.
    """
    rng = np.random.default_rng(seed)
    r0, r1 = r_range
    if radius is None:
        radius, length = drum_geometry(n, r_range, fill)
    else:
        length = 2.0 * radius
    V, T = drum_mesh(radius, length, n_theta, n_rings)
    inner = radius * math.cos(math.pi / n_theta)
    d = (2.0 * r1 + 0.02e-3) if nn_dist is None else nn_dist
    a = d * math.sqrt(2.0)
    margin = max(r1, 0.5 * d) + 0.01e-3
    lo = np.array([-0.5 * length + margin, -inner + margin, -inner + margin])
    hi = np.array([0.5 * length - margin, inner - margin, inner - margin])
    P = fcc_points(lo, hi, a)
    P = P[np.hypot(P[:, 1], P[:, 2]) <= inner - margin]
    if P.shape[0] < n:
        raise ValueError(f"drum holds only {P.shape[0]} lattice sites for {n} particles")
    order = np.lexsort((P[:, 0], P[:, 1], P[:, 2]))  # lowest first
    X = np.ascontiguousarray(P[order][:n])
    R = rng.uniform(r0, r1, size=n)
    v = rng.normal(scale=speed, size=(n, 3)) if speed > 0 else np.zeros((n, 3))
    w = np.zeros((n, 3))
    q = _unit_quaternions(rng, n)
    om = rpm * 2.0 * math.pi / 60.0
    params = base_params(dt=DT_DRUM, mu_s=0.4, mu_r=0.05, mu_t=0.05,
                         mesh_omega=(om, 0.0, 0.0), mesh_center=(0.0, 0.0, 0.0))
    params.update(over)
    dlo = np.array([-0.5 * length, -radius, -radius]) - 2 * r1
    dhi = np.array([0.5 * length, radius, radius]) + 2 * r1
    s = _scene("drum", seed, params, R, X, v, w, q, V, T, np.zeros(len(T)), (dlo, dhi))
    s["drum_radius"] = radius
    s["drum_length"] = length
    return s


def primitives_scene(n_side=(8, 8, 8), seed=6, spacing=1.96e-3, r_range=(0.9e-3, 1.1e-3),
                     jitter=2e-5, speed=0.02, spin=0.0, omega=0.0, **over):
    """Every kind of mesh element (Sec. 3.3) around and inside a particle lattice.

    A simple cubic lattice (as in lattice_box_scene, initial overlaps) in a box
    of six rectangles (one a rounded plate of radius 0.3 mm, set back by its
    radius), with obstacles placed on the lattice's interstitial lines and
    planes so that their nearest particles overlap them by at most ~0.1 mm:
      a capsule (segment, radius 0.35 mm) along x between two rows,
      a sphere (point, radius 0.7 mm) at the centre of a lattice cube,
      a triangle (radius 0) in the plane between two layers,
      a square plate (rectangle, radius 0.05 mm) across x between two columns.
    omega turns the whole mesh about the vertical axis through the box centre.
    Elements: 1 triangle, then 6 + 1 rectangles, 1 segment, 1 point.
    """
    rng = np.random.default_rng(seed)
    nx, ny, nz = n_side
    gi = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"),
                  axis=-1).reshape(-1, 3).astype(np.float64)
    n = gi.shape[0]
    R = rng.uniform(r_range[0], r_range[1], size=n)
    c0 = np.array([-0.5 * (nx - 1) * spacing, -0.5 * (ny - 1) * spacing, r_range[1]])
    X = gi * spacing + c0
    if jitter > 0:
        X += rng.uniform(-jitter, jitter, size=X.shape)
    v = rng.normal(scale=speed, size=(n, 3)) if speed > 0 else np.zeros((n, 3))
    w = rng.normal(scale=spin, size=(n, 3)) if spin > 0 else np.zeros((n, 3))
    q = _unit_quaternions(rng, n)

    def site(i, j, k):  # lattice coordinates -> position (half-integers allowed)
        return c0 + spacing * np.array([i, j, k], dtype=np.float64)

    lo = X.min(axis=0) - r_range[1] * 1.01
    hi = X.max(axis=0) + r_range[1] * 1.01
    lo[2] = 0.0
    Vb, _ = box_mesh(lo, hi)
    plate_r = 0.3e-3
    Vb[[1, 2, 5, 6], 0] += plate_r  # the +x face is the rounded plate, set back
    faces = [(0, 1, 2, 3), (4, 7, 6, 5), (0, 4, 5, 1), (1, 5, 6, 2), (2, 6, 7, 3), (3, 7, 4, 0)]
    verts = [*Vb]
    tri_v = [site(1.5, 1.5, 5.5), site(5.5, 2.5, 5.5), site(3.0, 5.5, 5.5)]
    ti = len(verts)
    verts += tri_v
    sq = [site(4.5, 2.0, 3.6), site(4.5, 5.0, 3.6), site(4.5, 5.0, 4.9), site(4.5, 2.0, 4.9)]
    ri = len(verts)
    verts += sq
    si = len(verts)
    verts += [site(1.2, 3.5, 2.5), site(5.8, 3.5, 2.5)]
    pi = len(verts)
    verts += [site(1.5, 5.5, 0.5)]
    V = np.array(verts, dtype=np.float64)
    T = np.array([[ti, ti + 1, ti + 2]], dtype=np.int32)
    E = [list(f) for f in faces] + [[ri, ri + 1, ri + 2, ri + 3], [si, si + 1, -1, -1],
                                    [pi, -1, -1, -1]]
    E = np.array(E, dtype=np.int32)
    er = np.zeros(len(E))
    er[3] = plate_r  # face (1, 5, 6, 2): +x
    er[6], er[7], er[8] = 0.05e-3, 0.35e-3, 0.7e-3
    centre = 0.5 * (lo + hi)
    params = base_params(dt=DT_BOX, mesh_omega=(0.0, 0.0, omega),
                         mesh_center=(centre[0], centre[1], 0.0))
    params.update(over)
    dlo = lo - 2 * r_range[1] - plate_r
    dhi = hi + 2 * r_range[1] + plate_r
    return _scene("primitives", seed, params, R, X, v, w, q, V, T, np.zeros(1), (dlo, dhi),
                  elems=E, elem_radius=er)


def eq_dt(rmin, rho, nu, E):
    """The paper's default time step (Eq. dt): R_min sqrt(rho (1 - nu^2) / E)."""
    return rmin * math.sqrt(rho * (1.0 - nu * nu) / E)


def _box_rect(x0, x1, y0, y1, z0, z1):
    """Vertices of an axis-aligned rectangle (one of the extents is zero), in order."""
    if x0 == x1:
        return [(x0, y0, z0), (x0, y1, z0), (x0, y1, z1), (x0, y0, z1)]
    if y0 == y1:
        return [(x0, y0, z0), (x1, y0, z0), (x1, y0, z1), (x0, y0, z1)]
    return [(x0, y0, z0), (x1, y0, z0), (x1, y1, z0), (x0, y1, z0)]


def repose_scene(n=20_000, seed=7, R=1.0e-3, gap_diameters=11, stream_diameters=6,
                 mu_s=3.0, mu_r=3.0, attempts=64, every=10, v0=-0.5, dt_div=10.0,
                 spawn_angle=60.0, **over):
    """Quasi-2D heap between two vertical plates (the piling example, Sec. 5).

    Monodisperse grains of radius R between plates gap_diameters diameters
    apart (y), with the material defaults of Table 2 (rho 1000, E 1 MPa, nu 0.3,
    e_n 0.5), the strong friction mu_s = mu_r = 3, mu_t = 2 mu_s / 3 (Table 2's
    default rule), and a time step dt_div = 10 times below Eq. dt.  As in the
    paper, a stream of spawned grains piles up: the spawn box spans the gap, is
    stream_diameters wide in x and sits above the height of the final heap for
    angles up to spawn_angle degrees; it gets `attempts` attempts every `every`
    steps, the grains start with vertical velocity v0, until n grains are in.
    The
    floor and the two end walls are far outside the heap's base.  All mesh
    elements are rectangles of radius 0.
    """
    d = 2.0 * R
    W = gap_diameters * d
    hy = 0.5 * W
    area = n * (math.pi / 6.0) * d ** 3 / (0.6 * W)  # heap cross-section at packing 0.6
    h60 = math.sqrt(area * math.tan(math.radians(60.0)))
    h_sp = math.sqrt(area * math.tan(math.radians(spawn_angle)))
    base40 = 2.0 * math.sqrt(area * math.tan(math.radians(40.0))) / math.tan(math.radians(40.0))
    half_floor = 0.8 * base40 + 5 * d
    z_sp = 1.1 * h_sp + 8 * d
    top = z_sp + 8 * d
    rects = [
        _box_rect(-half_floor, half_floor, -hy, hy, 0.0, 0.0),            # floor
        _box_rect(-half_floor, half_floor, -hy, -hy, 0.0, top),           # plate y-
        _box_rect(-half_floor, half_floor, hy, hy, 0.0, top),             # plate y+
        _box_rect(-half_floor, -half_floor, -hy, hy, 0.0, h60 + 4 * d),   # end wall x-
        _box_rect(half_floor, half_floor, -hy, hy, 0.0, h60 + 4 * d),     # end wall x+
    ]
    V = np.array([p for r in rects for p in r], dtype=np.float64)
    E = np.arange(4 * len(rects), dtype=np.int32).reshape(-1, 4)
    params = base_params(rho=1000.0, E=1.0e6, nu=0.3, e_n=0.5, mu_s=mu_s, mu_r=mu_r,
                         mu_t=2.0 * mu_s / 3.0, dt=eq_dt(R, 1000.0, 0.3, 1.0e6) / dt_div)
    params.update(over)
    half_stream = 0.5 * stream_diameters * d
    spawn = dict(n_max=n, lo=(-half_stream, -hy + R, z_sp), hi=(half_stream, hy - R, z_sp + 4 * d),
                 r_min=R, r_max=R, v0=(0.0, 0.0, v0), w0=(0.0, 0.0, 0.0), attempts=attempts,
                 every=every, seed=seed)
    lo = np.array([-half_floor, -hy, 0.0]) - 2 * d
    hi = np.array([half_floor, hy, top]) + 2 * d
    s = _scene("repose", seed, params, np.zeros(0), np.zeros((0, 3)), None, None, None, V, None,
               None, (lo, hi), elems=E, elem_radius=np.zeros(len(E)))
    s.update(gap=W, half_floor=half_floor, h60=h60, spawn=spawn, z_spawn=z_sp)
    return s
