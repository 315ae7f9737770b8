"""Python access to the FP64 DEM oracle (TEST INFRASTRUCTURE ONLY).

The oracle is a plain double-precision CPU restatement of the soft-sphere DEM
timestep of arXiv 2507.12610 (Sec. 2 and Sec. 3.2-3.3) with brute-force
O(N^2) pair search and O(N*M) particle-triangle search; see dem_oracle.cpp for
the readings it takes.  Only the tests, the smoke check and the CPU-baseline
leg of the benchmark may import this module.  It shares no code with the CUDA
library and never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_oracle.cpp")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.c_double
_I64 = ctypes.c_int64
_P = ctypes.c_void_p


class OracleSpawn(ctypes.Structure):
    """Spawning parameters (Sec. 3.1); layout of oracle_spawn."""
    _fields_ = [("n_max", _I64), ("lo", _D * 3), ("hi", _D * 3), ("r_min", _D), ("r_max", _D),
                ("v0", _D * 3), ("w0", _D * 3), ("attempts", ctypes.c_int32),
                ("every", ctypes.c_int32), ("seed", ctypes.c_uint64)]


def make_spawn(sp: dict) -> OracleSpawn:
    o = OracleSpawn()
    o.n_max = int(sp["n_max"])
    o.lo[:] = [float(c) for c in sp["lo"]]
    o.hi[:] = [float(c) for c in sp["hi"]]
    o.r_min, o.r_max = float(sp["r_min"]), float(sp["r_max"])
    o.v0[:] = [float(c) for c in sp.get("v0", (0.0, 0.0, 0.0))]
    o.w0[:] = [float(c) for c in sp.get("w0", (0.0, 0.0, 0.0))]
    o.attempts = int(sp["attempts"])
    o.every = int(sp.get("every", 1))
    o.seed = int(sp.get("seed", 0))
    return o


class OracleParams(ctypes.Structure):
    """Mirror of `oracle_params` in dem_oracle.cpp."""

    _fields_ = [
        ("E", _D), ("nu", _D), ("rho", _D), ("e_n", _D),
        ("mu_s", _D), ("mu_r", _D), ("mu_t", _D), ("eta", _D),
        ("g", _D * 3), ("dt", _D),
        ("mesh_omega", _D * 3), ("mesh_center", _D * 3),
        ("literal_sign", ctypes.c_int32), ("reserved", ctypes.c_int32),
    ]


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (g++, no FMA contraction)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["g++", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c++17",
               "-o", tmp, _SRC]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = ctypes.CDLL(_LIB)
    dp = ctypes.POINTER(_D)
    lib.oracle_create.restype = _P
    lib.oracle_create.argtypes = [ctypes.POINTER(OracleParams), _I64, dp, dp, dp, dp, dp,
                                  _I64, dp, _I64, ctypes.POINTER(ctypes.c_int32), dp]
    lib.oracle_destroy.argtypes = [_P]
    lib.oracle_step.argtypes = [_P, _I64]
    lib.oracle_read_state.argtypes = [_P, dp, dp, dp, dp]
    lib.oracle_read_forces.argtypes = [_P, dp, dp]
    lib.oracle_num_contacts.restype = _I64
    lib.oracle_num_contacts.argtypes = [_P]
    lib.oracle_degenerate.restype = _I64
    lib.oracle_degenerate.argtypes = [_P]
    lib.oracle_step_count.restype = _I64
    lib.oracle_step_count.argtypes = [_P]
    lib.oracle_read_contacts.argtypes = [_P, ctypes.POINTER(_I64), dp]
    lib.oracle_set_contacts.argtypes = [_P, _I64, ctypes.POINTER(_I64), dp]
    lib.oracle_set_step_count.argtypes = [_P, _I64]
    lib.oracle_set_state.argtypes = [_P, dp, dp, dp, dp]
    lib.oracle_read_coulomb.argtypes = [_P, dp]
    lib.oracle_closest_on_triangle.argtypes = [dp, dp, dp, dp, dp]
    lib.oracle_closest_on_element.argtypes = [dp, dp, ctypes.c_int32, dp]
    lib.oracle_beta.restype = _D
    lib.oracle_beta.argtypes = [_D]
    lib.oracle_contact_coeffs.argtypes = [ctypes.POINTER(OracleParams), ctypes.c_int32, _D, _D,
                                          _D, dp]
    lib.oracle_set_spawn.argtypes = [_P, ctypes.POINTER(OracleSpawn)]
    lib.oracle_set_materials.argtypes = [_P, ctypes.c_int32, dp, ctypes.POINTER(ctypes.c_int32)]
    lib.oracle_active.restype = _I64
    lib.oracle_active.argtypes = [_P]
    lib.oracle_capacity.restype = _I64
    lib.oracle_capacity.argtypes = [_P]
    lib.oracle_spawn_draws.restype = ctypes.c_uint64
    lib.oracle_spawn_draws.argtypes = [_P]
    lib.oracle_read_radii.argtypes = [_P, dp]
    lib.oracle_spawn_uniform.restype = _D
    lib.oracle_spawn_uniform.argtypes = [ctypes.c_uint64, ctypes.c_uint64]
    lib.oracle_sample_first_step.argtypes = [
        ctypes.POINTER(OracleParams), _I64, dp, dp, dp, dp, dp, _I64, dp, _I64,
        ctypes.POINTER(ctypes.c_int32), dp, _I64, _I64, ctypes.POINTER(_I64),
        dp, dp, dp, dp, dp, dp]
    _lib = lib
    return lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(_D))


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def elements(tris) -> np.ndarray:
    """Mesh elements as an (m, 4) int32 array of vertex indices padded with -1.

    Rows with 1, 2, 3 or 4 vertices are a point, a segment, a triangle or a
    rectangle (vertices in order around it).  (m, 3) triangle arrays are padded.
    """
    t = np.asarray(tris)
    if t.ndim == 1:
        t = t.reshape(-1, 3)
    out = np.full((t.shape[0], 4), -1, dtype=np.int32)
    out[:, :t.shape[1]] = t
    return np.ascontiguousarray(out)


def make_params(p: dict, literal_sign: bool = False) -> OracleParams:
    """Fill OracleParams from a plain dict (keys as in the scene generators)."""
    op = OracleParams()
    for k in ("E", "nu", "rho", "e_n", "mu_s", "mu_r", "mu_t", "eta", "dt"):
        setattr(op, k, float(p[k]))
    op.g[:] = [float(c) for c in p.get("g", (0.0, 0.0, 0.0))]
    op.mesh_omega[:] = [float(c) for c in p.get("mesh_omega", (0.0, 0.0, 0.0))]
    op.mesh_center[:] = [float(c) for c in p.get("mesh_center", (0.0, 0.0, 0.0))]
    op.literal_sign = 1 if literal_sign else 0
    return op


class OracleScene:
    """A DEM scene advanced by the FP64 oracle."""

    def __init__(self, params: dict, R, x, v=None, w=None, q=None, verts=None, tris=None,
                 tri_radius=None, literal_sign: bool = False, spawn=None, material=None,
                 material_mu=None):
        lib = _load()
        R = _f64(R, (-1,))
        n = R.shape[0]
        self.n = n
        x = _f64(x, (n, 3))
        v = _f64(np.zeros((n, 3)) if v is None else v, (n, 3))
        w = _f64(np.zeros((n, 3)) if w is None else w, (n, 3))
        if q is None:
            q = np.zeros((n, 4))
            q[:, 0] = 1.0
        q = _f64(q, (n, 4))
        self._p = make_params(params, literal_sign)
        if tris is None or len(tris) == 0:
            nv, nt = 0, 0
            vb = np.zeros(3)
            tb = np.full(4, -1, dtype=np.int32)
            rb = np.zeros(1)
        else:
            vb = _f64(verts, (-1, 3))
            tb = elements(tris)
            rb = _f64(np.zeros(len(tb)) if tri_radius is None else tri_radius, (-1,))
            nv, nt = vb.shape[0], tb.shape[0]
        self.n_tri = nt
        self._h = lib.oracle_create(ctypes.byref(self._p), n, _dptr(R), _dptr(x), _dptr(v),
                                    _dptr(w), _dptr(q), nv, _dptr(vb), nt,
                                    tb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                    _dptr(rb))
        self._lib = lib
        if material_mu is not None:
            # friction per material: (n_mat, 3) mu_s, mu_r, mu_t; material[i] per particle
            mu = _f64(material_mu, (-1, 3))
            mat = np.zeros(n, dtype=np.int32) if material is None else np.ascontiguousarray(
                np.asarray(material, dtype=np.int32).reshape(n))
            lib.oracle_set_materials(self._h, mu.shape[0], _dptr(mu),
                                     mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)))
        if spawn is not None:
            self._sp = make_spawn(spawn)
            lib.oracle_set_spawn(self._h, ctypes.byref(self._sp))
            self.n = int(lib.oracle_capacity(self._h))

    @property
    def active(self) -> int:
        """Particles taking part in the dynamics (rows 0 .. active-1)."""
        return int(self._lib.oracle_active(self._h))

    @property
    def spawn_draws(self) -> int:
        return int(self._lib.oracle_spawn_draws(self._h))

    def radii(self) -> np.ndarray:
        R = np.empty(self.n)
        self._lib.oracle_read_radii(self._h, _dptr(R))
        return R

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.oracle_destroy(h)
            self._h = None

    def step(self, nsteps: int = 1) -> None:
        self._lib.oracle_step(self._h, int(nsteps))

    @property
    def step_count(self) -> int:
        return int(self._lib.oracle_step_count(self._h))

    def set_step_count(self, c: int) -> None:
        self._lib.oracle_set_step_count(self._h, int(c))

    def state(self) -> dict:
        n = self.n
        x, v, w, q = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 4))
        self._lib.oracle_read_state(self._h, _dptr(x), _dptr(v), _dptr(w), _dptr(q))
        return {"x": x, "v": v, "w": w, "q": q}

    def forces(self):
        """Contact force and torque sums of the last step, (n,3) each."""
        F, T = np.empty((self.n, 3)), np.empty((self.n, 3))
        self._lib.oracle_read_forces(self._h, _dptr(F), _dptr(T))
        return F, T

    def contacts(self):
        """Active contacts after the last step: keys (m,2) int64 and history (m,7).

        keys[:,0] = i; keys[:,1] = j > i for a particle pair, or -1-k for triangle k.
        history columns: u_s (3), u_r (3), u_t.
        """
        m = int(self._lib.oracle_num_contacts(self._h))
        keys = np.empty((m, 2), dtype=np.int64)
        hist = np.empty((m, 7))
        if m:
            self._lib.oracle_read_contacts(self._h, keys.ctypes.data_as(ctypes.POINTER(_I64)),
                                           _dptr(hist))
        return keys, hist

    def set_contacts(self, keys, hist) -> None:
        keys = np.ascontiguousarray(np.asarray(keys, dtype=np.int64).reshape(-1, 2))
        hist = _f64(hist, (-1, 7))
        self._lib.oracle_set_contacts(self._h, keys.shape[0],
                                      keys.ctypes.data_as(ctypes.POINTER(_I64)), _dptr(hist))

    def set_state(self, x, v, w, q) -> None:
        """Replace x, v, w, q (caller order, all rows) with the given arrays."""
        n = self.n
        x, v, w, q = _f64(x, (n, 3)), _f64(v, (n, 3)), _f64(w, (n, 3)), _f64(q, (n, 4))
        self._lib.oracle_set_state(self._h, _dptr(x), _dptr(v), _dptr(w), _dptr(q))

    def coulomb(self) -> np.ndarray:
        """Coulomb ratios |f_m| / (mu_m |f_n|) (sliding, rolling, twisting) of
        the trial forces of the last step, rows in the order of contacts()."""
        m = int(self._lib.oracle_num_contacts(self._h))
        out = np.empty((m, 3))
        if m:
            self._lib.oracle_read_coulomb(self._h, _dptr(out))
        return out

    @property
    def degenerate(self) -> int:
        return int(self._lib.oracle_degenerate(self._h))


def closest_on_triangle(p, a, b, c) -> np.ndarray:
    lib = _load()
    p, a, b, c = (_f64(t, (3,)) for t in (p, a, b, c))
    out = np.empty(3)
    lib.oracle_closest_on_triangle(_dptr(p), _dptr(a), _dptr(b), _dptr(c), _dptr(out))
    return out


def closest_on_element(p, verts) -> np.ndarray:
    """Closest point on a point / segment / triangle / rectangle (1-4 vertices)."""
    lib = _load()
    p = _f64(p, (3,))
    v = _f64(verts, (-1, 3))
    out = np.empty(3)
    lib.oracle_closest_on_element(_dptr(p), _dptr(v), v.shape[0], _dptr(out))
    return out


def beta(e_n: float) -> float:
    return float(_load().oracle_beta(float(e_n)))


def contact_coeffs(params: dict, Ri: float, Rj: float, delta: float, wall: bool = False) -> dict:
    """Effective properties and coefficients the oracle uses for one contact."""
    lib = _load()
    p = make_params(params)
    out = np.empty(8)
    lib.oracle_contact_coeffs(ctypes.byref(p), 1 if wall else 0, float(Ri), float(Rj),
                              float(delta), _dptr(out))
    return dict(zip(("Es", "Gs", "Rs", "ms", "kn", "ks", "cn", "cs"), out.tolist()))


def sample_first_step(params: dict, R, x, v, w, q, verts, tris, tri_radius, ids,
                      step_index: int = 0, literal_sign: bool = False) -> dict:
    """First step (no contact history) for a sample of particles, one by one.

    Returns the contact sums F, T and the integrated x, v, w, q of the sampled
    particles, rows in the order of `ids`.
    """
    lib = _load()
    R = _f64(R, (-1,))
    n = R.shape[0]
    x, v, w = _f64(x, (n, 3)), _f64(v, (n, 3)), _f64(w, (n, 3))
    q = _f64(q, (n, 4))
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
    ns = ids.shape[0]
    if tris is None or len(tris) == 0:
        vb, tb, rb, nv, nt = np.zeros(3), np.full(4, -1, dtype=np.int32), np.zeros(1), 0, 0
    else:
        vb = _f64(verts, (-1, 3))
        tb = elements(tris)
        rb = _f64(np.zeros(len(tb)) if tri_radius is None else tri_radius, (-1,))
        nv, nt = vb.shape[0], tb.shape[0]
    p = make_params(params, literal_sign)
    out = {k: np.empty((ns, 3)) for k in ("F", "T", "x", "v", "w")}
    out["q"] = np.empty((ns, 4))
    lib.oracle_sample_first_step(ctypes.byref(p), n, _dptr(R), _dptr(x), _dptr(v), _dptr(w),
                                 _dptr(q), nv, _dptr(vb), nt,
                                 tb.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)), _dptr(rb),
                                 int(step_index), ns,
                                 ids.ctypes.data_as(ctypes.POINTER(_I64)),
                                 _dptr(out["F"]), _dptr(out["T"]), _dptr(out["x"]),
                                 _dptr(out["v"]), _dptr(out["w"]), _dptr(out["q"]))
    return out


def spawn_uniform(seed: int, k: int) -> float:
    """k-th uniform of the spawn stream (SplitMix64, top 53 bits)."""
    return float(_load().oracle_spawn_uniform(int(seed), int(k)))
