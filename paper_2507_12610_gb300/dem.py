"""Thin Python binding of libdem (include/dem.h).

Argument marshalling only: every step of the DEM path runs in the CUDA
library.  The functions keep the C names; `Scene` is a small convenience
wrapper that owns a `dem_scene*`.  PyTorch is used only to hand the library
the current CUDA stream.  If the compiled library is missing this module
raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("DEM_LIB_PATH") or os.path.join(HERE, "libdem.so")

DEM_OK = 0
DEM_ERR_INVALID = 1
DEM_ERR_CAPACITY = 2
DEM_ERR_NONFINITE = 3
DEM_ERR_TIMEOUT = 4
DEM_ERR_CUDA = 5
DEM_ERR_NOMEM = 6

DEM_FP64 = 0
DEM_MIXED = 1
DEM_MIXED64 = 2

_D = ctypes.c_double
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_DP = ctypes.POINTER(ctypes.c_double)

# every symbol declared in include/dem.h
EXPORTS = ("dem_scene_create", "dem_step", "dem_synchronize", "dem_read_state",
           "dem_read_forces", "dem_read_contacts", "dem_get_stats", "dem_save", "dem_load",
           "dem_scene_destroy", "dem_status_string", "dem_step_timed",
           "dem_contact_forces_noalloc", "dem_read_radii", "dem_probe_fp64_fma",
           "dem_scene_create_with_allocator")

# dem_alloc_fn / dem_free_fn
ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p)


class dem_params(ctypes.Structure):
    _fields_ = [("E", _D), ("nu", _D), ("rho", _D), ("e_n", _D), ("mu_s", _D), ("mu_r", _D),
                ("mu_t", _D), ("eta", _D), ("g", _D * 3), ("dt", _D),
                ("mesh_omega", _D * 3), ("mesh_center", _D * 3), ("skin", _D),
                ("domain_lo", _D * 3), ("domain_hi", _D * 3), ("precision", _I32),
                ("max_neighbors", _I32), ("max_mesh_contacts", _I32),
                ("record_forces", _I32), ("n_max", _I64), ("spawn_lo", _D * 3),
                ("spawn_hi", _D * 3), ("spawn_r_min", _D), ("spawn_r_max", _D),
                ("spawn_v0", _D * 3), ("spawn_w0", _D * 3), ("spawn_attempts", _I32),
                ("spawn_every", _I32), ("spawn_seed", ctypes.c_uint64),
                ("step_warps", _I32), ("reserved", _I32)]


class dem_particles(ctypes.Structure):
    _fields_ = [("n", _I64), ("R", _DP), ("x", _DP), ("v", _DP), ("w", _DP), ("q", _DP),
                ("n_materials", _I32), ("material", ctypes.POINTER(ctypes.c_int32)),
                ("material_mu", _DP)]


class dem_mesh(ctypes.Structure):
    _fields_ = [("n_vert", _I64), ("vert", _DP), ("n_tri", _I64),
                ("tri", ctypes.POINTER(ctypes.c_int32)), ("tri_radius", _DP),
                ("n_elem", _I64), ("elem", ctypes.POINTER(ctypes.c_int32)),
                ("elem_radius", _DP)]


class dem_stats(ctypes.Structure):
    _fields_ = [("steps", _I64), ("rebuilds", _I64), ("pair_contacts", _I64),
                ("mesh_contacts", _I64), ("list_entries", _I64), ("mesh_candidates", _I64),
                ("max_list_len", _I32), ("status", _I32), ("launches_per_step", _I32),
                ("launches_per_rebuild", _I32), ("active", _I64), ("capacity", _I64)]


class DemError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        super().__init__(f"{what}: {status_string(code)} ({code})")


_lib = None


def load(path: str = LIB_PATH):
    """Load libdem.so; raises if it has not been built (no CPU fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libdem.so not built at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P = ctypes.c_void_p
    lib.dem_scene_create.argtypes = [ctypes.POINTER(dem_params), ctypes.POINTER(dem_particles),
                                     ctypes.POINTER(dem_mesh), P, ctypes.POINTER(P)]
    lib.dem_scene_create_with_allocator.argtypes = [
        ctypes.POINTER(dem_params), ctypes.POINTER(dem_particles), ctypes.POINTER(dem_mesh), P,
        ALLOC_FN, FREE_FN, P, ctypes.POINTER(P)]
    lib.dem_step.argtypes = [P, _I64]
    lib.dem_synchronize.argtypes = [P]
    lib.dem_step_timed.argtypes = [P, _I64, _DP]
    lib.dem_read_state.argtypes = [P, _DP, _DP, _DP, _DP]
    lib.dem_read_forces.argtypes = [P, _DP, _DP]
    lib.dem_read_contacts.argtypes = [P, _I64, ctypes.POINTER(_I64), _DP, ctypes.POINTER(_I64)]
    lib.dem_get_stats.argtypes = [P, ctypes.POINTER(dem_stats)]
    lib.dem_save.argtypes = [P, P, ctypes.POINTER(ctypes.c_size_t)]
    lib.dem_load.argtypes = [P, P, ctypes.c_size_t]
    lib.dem_contact_forces_noalloc.argtypes = [ctypes.POINTER(dem_params), _I64, _D, P, P, P,
                                               P, P, P, P]
    lib.dem_probe_fp64_fma.argtypes = [_I64, P, _DP]
    lib.dem_scene_destroy.argtypes = [P]
    lib.dem_scene_destroy.restype = None
    lib.dem_status_string.argtypes = [ctypes.c_int]
    lib.dem_status_string.restype = ctypes.c_char_p
    for name in EXPORTS:
        if name not in ("dem_scene_destroy", "dem_status_string"):
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def status_string(code: int) -> str:
    return load().dem_status_string(int(code)).decode()


def _check(rc: int, what: str):
    if rc != DEM_OK:
        raise DemError(rc, what)


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


def _p(a):
    return None if a is None else a.ctypes.data_as(_DP)


def make_params(p: dict, precision: int = DEM_FP64, skin: float = 0.0, max_neighbors: int = 0,
                max_mesh_contacts: int = 0, record_forces: bool = False,
                domain=None, spawn=None, step_warps: int = 0) -> dem_params:
    """dem_params from a parameter dict; `spawn` (optional) is a dict with
    n_max, lo, hi, r_min, r_max, v0, w0, attempts, every, seed (Sec. 3.1)."""
    dp = dem_params()
    for k in ("E", "nu", "rho", "e_n", "mu_s", "mu_r", "mu_t", "eta", "dt"):
        setattr(dp, k, float(p[k]))
    dp.g[:] = [float(c) for c in p.get("g", (0, 0, 0))]
    dp.mesh_omega[:] = [float(c) for c in p.get("mesh_omega", (0, 0, 0))]
    dp.mesh_center[:] = [float(c) for c in p.get("mesh_center", (0, 0, 0))]
    dp.skin = float(skin)
    if domain is not None:
        dp.domain_lo[:] = [float(c) for c in domain[0]]
        dp.domain_hi[:] = [float(c) for c in domain[1]]
    dp.precision = int(precision)
    dp.max_neighbors = int(max_neighbors)
    dp.max_mesh_contacts = int(max_mesh_contacts)
    dp.record_forces = 1 if record_forces else 0
    dp.step_warps = int(step_warps)
    if spawn is not None:
        dp.n_max = int(spawn["n_max"])
        dp.spawn_lo[:] = [float(c) for c in spawn["lo"]]
        dp.spawn_hi[:] = [float(c) for c in spawn["hi"]]
        dp.spawn_r_min = float(spawn["r_min"])
        dp.spawn_r_max = float(spawn["r_max"])
        dp.spawn_v0[:] = [float(c) for c in spawn.get("v0", (0.0, 0.0, 0.0))]
        dp.spawn_w0[:] = [float(c) for c in spawn.get("w0", (0.0, 0.0, 0.0))]
        dp.spawn_attempts = int(spawn["attempts"])
        dp.spawn_every = int(spawn.get("every", 1))
        dp.spawn_seed = int(spawn.get("seed", 0))
    return dp


def contact_forces_noalloc(params: dict, n: int, r_max: float, R_ptr: int, x_ptr: int,
                           v_ptr: int, w_ptr: int, F_ptr: int, T_ptr: int, domain,
                           stream=None) -> int:
    """dem_contact_forces_noalloc on caller-owned device buffers (raw pointers).

    The library allocates nothing for this call; see include/dem.h for the
    limits and the set-up made by the first call on a device.
    """
    lib = load()
    dp = make_params(params, domain=domain)
    st = stream if stream is not None else current_stream()
    return int(lib.dem_contact_forces_noalloc(ctypes.byref(dp), int(n), float(r_max), R_ptr,
                                              x_ptr, v_ptr, w_ptr, F_ptr, T_ptr, st))


def probe_fp64_fma(iters: int = 16384, stream=None) -> float:
    """FP64 FMA throughput of the current device (FMAs per second)."""
    lib = load()
    out = _D(0.0)
    st = stream if stream is not None else current_stream()
    _check(lib.dem_probe_fp64_fma(int(iters), st, ctypes.byref(out)), "dem_probe_fp64_fma")
    return out.value


def current_stream():
    """The current torch CUDA stream as a cudaStream_t (None if torch is absent)."""
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


class TorchAllocator:
    """Device memory for scenes from PyTorch's caching allocator, handed to
    dem_scene_create_with_allocator (the blocks count in
    torch.cuda.memory_allocated and return to torch's pool when the scene is
    destroyed).  `live` maps each block the library holds to its size."""

    def __init__(self, device=None, stream=None):
        import torch
        self._torch = torch
        self.device = torch.cuda.current_device() if device is None else device
        self.stream = stream
        self.live = {}
        self.alloc_fn = ALLOC_FN(self._alloc)
        self.free_fn = FREE_FN(self._free)

    def _alloc(self, nbytes, ctx):
        try:
            p = self._torch.cuda.caching_allocator_alloc(int(nbytes), self.device, self.stream)
        except RuntimeError:  # out of memory: the library reports DEM_ERR_NOMEM
            return None
        self.live[int(p)] = int(nbytes)
        return p

    def _free(self, ptr, ctx):
        self.live.pop(int(ptr), None)
        self._torch.cuda.caching_allocator_delete(ptr)


class Scene:
    """Owner of one `dem_scene*` created from host arrays."""

    def __init__(self, params: dict, R, x, v=None, w=None, q=None, verts=None, tris=None,
                 tri_radius=None, elems=None, elem_radius=None,
                 precision: int = DEM_FP64, skin: float = 0.0,
                 max_neighbors: int = 0, max_mesh_contacts: int = 0,
                 record_forces: bool = False, domain=None, stream=None, spawn=None,
                 material=None, material_mu=None, step_warps: int = 0, allocator=None):
        lib = load()
        self._lib = lib
        self._h = ctypes.c_void_p()
        # kept for regrow(): the same scene with larger list capacities
        self._init_args = (params, R, x, v, w, q, verts, tris, tri_radius, elems, elem_radius)
        self._init_kw = dict(precision=precision, skin=skin, max_neighbors=max_neighbors,
                             max_mesh_contacts=max_mesh_contacts, record_forces=record_forces,
                             domain=domain, stream=stream, spawn=spawn, material=material,
                             material_mu=material_mu, step_warps=step_warps,
                             allocator=allocator)
        R = _f64(R, (-1,))
        n = R.shape[0]
        # rows: the given particles, then (with spawning) inactive rows up to n_max
        self.n = max(n, int(spawn["n_max"])) if spawn is not None else n
        x = _f64(x, (n, 3))
        v = None if v is None else _f64(v, (n, 3))
        w = None if w is None else _f64(w, (n, 3))
        q = None if q is None else _f64(q, (n, 4))
        self.precision = precision
        self._pp = make_params(params, precision, skin, max_neighbors, max_mesh_contacts,
                               record_forces, domain, spawn, step_warps)
        pa = dem_particles(n, _p(R), _p(x), _p(v), _p(w), _p(q))
        keep = [R, x, v, w, q]
        if material_mu is not None:
            # friction per material: (n_mat, 3) mu_s, mu_r, mu_t; material[i] per particle
            mu = _f64(material_mu, (-1, 3))
            mat = None if material is None else np.ascontiguousarray(
                np.asarray(material, dtype=np.int32).reshape(n))
            pa.n_materials = mu.shape[0]
            pa.material_mu = _p(mu)
            if mat is not None:
                pa.material = mat.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
            keep += [mu, mat]
        me = dem_mesh()
        has_tris = tris is not None and len(tris) > 0
        has_elems = elems is not None and len(elems) > 0
        if has_tris or has_elems:
            # elements: the triangles, then the rows of `elems` (1-4 vertex
            # indices padded with -1: point, segment, triangle, rectangle)
            i32p = ctypes.POINTER(ctypes.c_int32)
            V = _f64(verts, (-1, 3))
            T = np.ascontiguousarray(np.asarray(tris if has_tris else np.zeros((0, 3)),
                                                dtype=np.int32).reshape(-1, 3))
            Rt = None if tri_radius is None else _f64(tri_radius, (-1,))
            El = np.ascontiguousarray(np.asarray(elems if has_elems else np.zeros((0, 4)),
                                                 dtype=np.int32).reshape(-1, 4))
            Re = None if elem_radius is None else _f64(elem_radius, (-1,))
            me = dem_mesh(V.shape[0], _p(V), T.shape[0], T.ctypes.data_as(i32p), _p(Rt),
                          El.shape[0], El.ctypes.data_as(i32p), _p(Re))
            keep += [V, T, Rt, El, Re]
        self.n_tri = me.n_tri + me.n_elem  # mesh elements (triangles first)
        st = stream if stream is not None else current_stream()
        # the allocator's callbacks must outlive the scene (they free its blocks)
        self._allocator = allocator
        if allocator is None:
            rc = lib.dem_scene_create(ctypes.byref(self._pp), ctypes.byref(pa), ctypes.byref(me),
                                      st, ctypes.byref(self._h))
        else:
            rc = lib.dem_scene_create_with_allocator(
                ctypes.byref(self._pp), ctypes.byref(pa), ctypes.byref(me), st,
                allocator.alloc_fn, allocator.free_fn, None, ctypes.byref(self._h))
        del keep
        _check(rc, "dem_scene_create")

    @classmethod
    def from_dict(cls, s: dict, **kw):
        kw.setdefault("spawn", s.get("spawn"))
        kw.setdefault("material", s.get("material"))
        kw.setdefault("material_mu", s.get("material_mu"))
        return cls(s["params"], s["R"], s["x"], s.get("v"), s.get("w"), s.get("q"),
                   s.get("verts"), s.get("tris"), s.get("tri_radius"), s.get("elems"),
                   s.get("elem_radius"), **kw)

    @property
    def R(self) -> np.ndarray:
        """Radii of all rows (0 for rows awaiting spawning)."""
        return self.radii()

    def radii(self) -> np.ndarray:
        R = np.empty(self.n)
        _check(self._lib.dem_read_radii(self._h, _p(R)), "dem_read_radii")
        return R

    @property
    def active(self) -> int:
        return int(self.stats()["active"])

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.dem_scene_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int = 1):
        _check(self._lib.dem_step(self._h, int(nsteps)), "dem_step")

    # list capacities the library accepts (include/dem.h)
    MAX_NEIGHBORS, MAX_MESH_CONTACTS = 64, 255

    def regrow(self, factor: int = 2) -> None:
        """Answer DEM_ERR_CAPACITY: the same scene with `factor` times the list
        capacities (up to the library's limits), continuing from the last
        completed step.  The step that overflowed did no work, so its state
        and friction history are saved (dem_save), a scene with the larger
        capacities is created and the blob loaded into it (dem_load)."""
        blob = self.save()
        kw = dict(self._init_kw)
        cap = kw["max_neighbors"] if kw["max_neighbors"] > 0 else self.MAX_NEIGHBORS
        capm = kw["max_mesh_contacts"] if kw["max_mesh_contacts"] > 0 else 16
        kw["max_neighbors"] = min(self.MAX_NEIGHBORS, factor * cap)
        kw["max_mesh_contacts"] = min(self.MAX_MESH_CONTACTS, factor * capm)
        if (kw["max_neighbors"], kw["max_mesh_contacts"]) == (cap, capm):
            raise DemError(DEM_ERR_CAPACITY, "regrow: capacities at the library's limit")
        self.close()
        self.__init__(*self._init_args, **kw)
        self.load(blob)

    def step_regrowing(self, nsteps: int, chunk: int = 256, max_regrows: int = 8) -> int:
        """dem_step in chunks of `chunk` steps, checking the status after each;
        a list overflow (DEM_ERR_CAPACITY) is answered by regrow() and the
        steps that did no work are taken again.  Other errors raise.  Returns
        the number of regrows."""
        start = self.stats()["steps"]
        regrows = 0
        while True:
            done = self.stats()["steps"] - start
            if done >= nsteps:
                return regrows
            self.step(min(chunk, nsteps - done))
            rc = self.synchronize()
            if rc == DEM_ERR_CAPACITY:
                if regrows >= max_regrows:
                    raise DemError(rc, "step_regrowing: too many regrows")
                self.regrow()
                regrows += 1
            elif rc != DEM_OK:
                raise DemError(rc, "dem_step")

    def step_timed(self, nsteps: int) -> np.ndarray:
        """Run nsteps phase by phase; device ms of [mesh pose, rebuild, step, advance]."""
        ms = np.zeros(4)
        _check(self._lib.dem_step_timed(self._h, int(nsteps), _p(ms)), "dem_step_timed")
        return ms

    def synchronize(self) -> int:
        return int(self._lib.dem_synchronize(self._h))

    def state(self) -> dict:
        n = self.n
        x, v, w, q = np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 3)), np.empty((n, 4))
        _check(self._lib.dem_read_state(self._h, _p(x), _p(v), _p(w), _p(q)), "dem_read_state")
        return {"x": x, "v": v, "w": w, "q": q}

    def read_state_into(self, x, v, w, q) -> int:
        return int(self._lib.dem_read_state(self._h, _p(x), _p(v), _p(w), _p(q)))

    def forces(self):
        F, T = np.empty((self.n, 3)), np.empty((self.n, 3))
        _check(self._lib.dem_read_forces(self._h, _p(F), _p(T)), "dem_read_forces")
        return F, T

    def contacts(self):
        cnt = _I64(0)
        rc = self._lib.dem_read_contacts(self._h, 0, None, None, ctypes.byref(cnt))
        if rc not in (DEM_OK, DEM_ERR_CAPACITY):
            _check(rc, "dem_read_contacts")
        m = cnt.value
        keys = np.empty((m, 2), dtype=np.int64)
        hist = np.empty((m, 7))
        _check(self._lib.dem_read_contacts(self._h, m, keys.ctypes.data_as(ctypes.POINTER(_I64)),
                                           _p(hist), ctypes.byref(cnt)), "dem_read_contacts")
        return keys, hist

    def stats(self) -> dict:
        st = dem_stats()
        _check(self._lib.dem_get_stats(self._h, ctypes.byref(st)), "dem_get_stats")
        return {k: getattr(st, k) for k, _ in dem_stats._fields_}

    def save(self) -> bytes:
        ln = ctypes.c_size_t(0)
        _check(self._lib.dem_save(self._h, None, ctypes.byref(ln)), "dem_save")
        buf = ctypes.create_string_buffer(ln.value)
        _check(self._lib.dem_save(self._h, buf, ctypes.byref(ln)), "dem_save")
        return buf.raw[:ln.value]

    def load(self, blob: bytes):
        buf = ctypes.create_string_buffer(blob, len(blob))
        _check(self._lib.dem_load(self._h, buf, len(blob)), "dem_load")
