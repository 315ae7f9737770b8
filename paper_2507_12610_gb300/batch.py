"""Batched ensembles: many independent scenes advanced as one scene.

Each scene keeps its own particles, mesh and friction coefficients; the
scenes are packed side by side in space with gaps wider than any contact
reach, so no contact ever joins two of them, and the whole batch runs as one
`dem.Scene`: every kernel of a step covers all scenes at once and a step is
one CUDA-graph replay for the whole ensemble.  A scene's friction is its
material (one material per scene).

The workload here is hopper discharge: a conical funnel of 256 triangles
(32 facets around, 4 rings) with its outlet open, a closed catch box below
it, and particles filling the funnel from the bottom on a cubic lattice.
This module builds inputs and reads results; it holds none of the contact or
integration arithmetic.
"""
from __future__ import annotations

import math
import time

import numpy as np

from . import scenes

# tile spacing: wider than two particle diameters plus any skin
GAP = 0.01


def funnel_mesh(r_out, r_top, height, z0, n_theta=32, n_rings=4):
    """Side of a conical funnel (frustum) about the vertical axis through the
    origin, outlet radius r_out at height z0, top radius r_top at z0 + height:
    n_rings x n_theta quads, two triangles each (256 for 32 x 4)."""
    th = 2.0 * math.pi * np.arange(n_theta) / n_theta
    V = []
    for k in range(n_rings + 1):
        f = k / n_rings
        r = r_out + f * (r_top - r_out)
        z = z0 + f * height
        V += [(r * math.cos(t), r * math.sin(t), z) for t in th]
    T = []
    for k in range(n_rings):
        for i in range(n_theta):
            a = k * n_theta + i
            b = k * n_theta + (i + 1) % n_theta
            c = (k + 1) * n_theta + i
            d = (k + 1) * n_theta + (i + 1) % n_theta
            T += [(a, b, d), (a, d, c)]
    return np.array(V, dtype=np.float64), np.array(T, dtype=np.int32)


def hopper_scene(n, seed, mu=(0.5, 0.1, 0.1), r_range=(0.9e-3, 1.1e-3),
                 half_angle_deg=30.0, outlet_diameters=10.0, pitch_factor=2.05, n_theta=32,
                 n_rings=4):
    """One hopper-discharge scene: particles on a lattice (pitch pitch_factor
    R_max; below 2 the spheres start overlapping) in a conical funnel of
    2 n_theta n_rings triangles, sized to hold n, above an open outlet, and a
    catch box below.  Returns a scene dict (particles, triangles, rectangles,
    mu)."""
    rng = np.random.default_rng(seed)
    rmax = r_range[1]

    def drop_of(h):  # outlet height above the catch floor
        return 0.5 * h + 0.02

    pitch = pitch_factor * rmax
    r_out = 0.5 * outlet_diameters * 2 * rmax
    ta = math.tan(math.radians(half_angle_deg))
    # the lowest funnel (this shape) whose lattice points, kept R_max (normal
    # to the wall) inside, hold n
    cosa = math.cos(math.radians(half_angle_deg))
    H = max(0.01, (n * pitch ** 3 * 1.2 * 3.0 / (math.pi * ta * ta)) ** (1.0 / 3.0) - r_out / ta)
    while True:
        r_top = r_out + H * ta
        m = int(math.ceil(r_top / pitch)) + 1
        nz = int(math.ceil(H / pitch))
        g = np.stack(np.meshgrid(np.arange(-m, m + 1), np.arange(-m, m + 1), np.arange(nz),
                                 indexing="ij"), -1).reshape(-1, 3).astype(np.float64)
        P = np.empty_like(g)
        P[:, :2] = g[:, :2] * pitch
        P[:, 2] = drop_of(H) + 0.5 * pitch + g[:, 2] * pitch
        rad = np.hypot(P[:, 0], P[:, 1])
        r_at = r_out + (P[:, 2] - drop_of(H)) * ta
        inside = (rad + rmax / cosa + 0.2 * rmax <= r_at) & (P[:, 2] + rmax <= drop_of(H) + H)
        P = P[inside]
        if P.shape[0] >= n:
            break
        H *= 1.05
    drop = drop_of(H)
    z_out = drop
    V, T = funnel_mesh(r_out, r_top, H, z_out, n_theta, n_rings)
    P = P[np.lexsort((P[:, 0], P[:, 1], P[:, 2]))][:n]
    R = rng.uniform(r_range[0], r_range[1], size=n)
    v = rng.normal(scale=0.01, size=(n, 3))
    w = np.zeros((n, 3))
    q = scenes._unit_quaternions(rng, n)
    # catch box: floor and four walls around the funnel's footprint
    half = r_top + 2 * pitch
    top = z_out - 0.25 * drop
    rects = [scenes._box_rect(-half, half, -half, half, 0.0, 0.0),
             scenes._box_rect(-half, -half, -half, half, 0.0, top),
             scenes._box_rect(half, half, -half, half, 0.0, top),
             scenes._box_rect(-half, half, -half, -half, 0.0, top),
             scenes._box_rect(-half, half, half, half, 0.0, top)]
    nv = V.shape[0]
    V = np.vstack([V, np.array([p for r in rects for p in r])])
    El = (nv + np.arange(4 * len(rects))).reshape(-1, 4).astype(np.int32)
    lo = np.array([-half, -half, 0.0])
    hi = np.array([half, half, z_out + H])
    return dict(n=n, R=R, x=P, v=v, w=w, q=q, verts=V, tris=T, elems=El, mu=tuple(mu),
                box=(lo, hi), z_outlet=z_out)


def ensemble(n_scenes=512, seed=11, n_range=(500, 20_000), mu_s=(0.2, 0.8), mu_r=(0.0, 0.2),
             mu_t=(0.0, 0.2)):
    """The batched-ensemble workload: n_scenes hoppers with particle counts
    log-uniform in n_range and friction coefficients uniform in the given
    ranges, one seed per scene."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(math.log(n_range[0]), math.log(n_range[1]), n_scenes)).astype(int)
    mus = np.stack([rng.uniform(*mu_s, n_scenes), rng.uniform(*mu_r, n_scenes),
                    rng.uniform(*mu_t, n_scenes)], axis=1)
    return [hopper_scene(int(n), seed * 100003 + k, tuple(mus[k])) for k, n in enumerate(ns)]


def pack(boxes, gap=GAP):
    """Offsets placing boxes (lo, hi) side by side without overlap, gap apart:
    shelves along x in rows along y in layers along z, tallest first."""
    size = np.array([np.asarray(hi) - np.asarray(lo) for lo, hi in boxes]) + gap
    order = np.argsort(-size[:, 2], kind="stable")
    total = float(np.sum(size[:, 0] * size[:, 1] * size[:, 2]))
    side = max(total ** (1.0 / 3.0), float(size[:, 0].max()), float(size[:, 1].max()))
    off = np.zeros((len(boxes), 3))
    x = y = z = 0.0
    row_d = layer_h = 0.0
    for k in order:
        sx, sy, sz = size[k]
        if x > 0 and x + sx > side:
            x, y = 0.0, y + row_d
            row_d = 0.0
        if y > 0 and y + sy > side:
            x, y, z = 0.0, 0.0, z + layer_h
            row_d = layer_h = 0.0
        off[k] = np.array([x, y, z]) - np.asarray(boxes[k][0])
        x += sx
        row_d = max(row_d, sy)
        layer_h = max(layer_h, sz)
    return off


def combine(scene_list, params=None, gap=GAP):
    """One scene dict for a list of hopper scenes: particles concatenated
    (scene k's particles take material k), meshes concatenated (triangles,
    then the rectangles of all scenes), each scene shifted by its packing
    offset.  Also returns per-scene particle ranges and offsets."""
    off = pack([s["box"] for s in scene_list], gap)
    R, X, Vv, W, Q, mat = [], [], [], [], [], []
    verts, tris, elems = [], [], []
    nvert = 0
    ranges = []
    start = 0
    for k, s in enumerate(scene_list):
        R.append(s["R"])
        X.append(s["x"] + off[k])
        Vv.append(s["v"])
        W.append(s["w"])
        Q.append(s["q"])
        mat.append(np.full(len(s["R"]), k, dtype=np.int32))
        verts.append(s["verts"] + off[k])
        tris.append(s["tris"] + nvert)
        elems.append(s["elems"] + nvert)
        nvert += s["verts"].shape[0]
        ranges.append((start, start + len(s["R"])))
        start += len(s["R"])
    p = scenes.base_params(rho=2500.0, e_n=0.5, dt=scenes.DT_BOX)
    if params:
        p.update(params)
    return dict(params=p, R=np.concatenate(R), x=np.vstack(X), v=np.vstack(Vv),
                w=np.vstack(W), q=np.vstack(Q), verts=np.vstack(verts), tris=np.vstack(tris),
                tri_radius=None, elems=np.vstack(elems), elem_radius=None,
                material=np.concatenate(mat),
                material_mu=np.array([s["mu"] for s in scene_list], dtype=np.float64),
                ranges=ranges, offsets=off, z_outlet=np.array([s["z_outlet"] for s in scene_list]))


def discharged(batch, x):
    """Fraction of each scene's particles below its funnel outlet."""
    out = []
    for k, (a, b) in enumerate(batch["ranges"]):
        z = x[a:b, 2] - batch["offsets"][k, 2]
        out.append(float(np.mean(z < batch["z_outlet"][k])))
    return np.array(out)


def autotune(batch, precision=1, skins=None, block_warps=(4, 8), steps=200, warmup=50,
             dem=None):
    """Pick the list skin and the step kernel's warps per block by timing
    short runs of the batch itself (device time per step, CUDA events around
    whole graph replays).  Returns (best, table)."""
    if dem is None:
        from . import dem
    rmax = float(np.max(batch["R"]))
    skins = skins or [0.1 * rmax, 0.2 * rmax, 0.35 * rmax, 0.5 * rmax]
    table = []
    for sk in skins:
        for bw in block_warps:
            sc = dem.Scene.from_dict(batch, precision=precision, skin=sk, step_warps=bw)
            sc.step(warmup)
            sc.synchronize()
            t0 = time.perf_counter()
            sc.step(steps)
            sc.synchronize()
            ms = (time.perf_counter() - t0) * 1e3 / steps
            table.append({"skin": sk, "step_warps": bw, "ms_per_step": ms,
                          "rebuilds": sc.stats()["rebuilds"]})
            sc.close()
    best = min(table, key=lambda r: r["ms_per_step"])
    return best, table
