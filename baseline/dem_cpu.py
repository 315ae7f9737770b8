"""CPU baseline of the DEM timestep in the design of the paper's own program.

`dem_cpu.cpp` (beside this file) is a double-precision OpenMP program with
the structure the paper describes for its C++ code (Sec. 3 and Sec. 5):
linked cells of edge 2 R_max over the ensemble's bounding box rebuilt every
step, one evaluation per particle pair, per-particle contact lists with an
active flag, OpenMP over particles and mesh elements.  It is timed beside the
GPU library by `bench.py` on the same workloads.  It shares no code with the
CUDA library or the test oracle.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "dem_cpu.cpp")
_LIB = os.path.join(_HERE, "libdem_cpu.so")
_lock = threading.Lock()
_lib = None
_D = ctypes.c_double
_DP = ctypes.POINTER(_D)


class dcpu_params(ctypes.Structure):
    _fields_ = [("E", _D), ("nu", _D), ("rho", _D), ("e_n", _D), ("mu_s", _D), ("mu_r", _D),
                ("mu_t", _D), ("eta", _D), ("g", _D * 3), ("dt", _D), ("mesh_omega", _D * 3),
                ("mesh_center", _D * 3)]


def build(force: bool = False) -> str:
    """Compile libdem_cpu.so next to its source (g++ -O3 -fopenmp)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["g++", "-O3", "-fopenmp", "-fPIC", "-shared", "-std=c++17", "-o", tmp,
                        _SRC], check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        lib.dcpu_create.restype = P
        lib.dcpu_create.argtypes = [ctypes.POINTER(dcpu_params), ctypes.c_int64, _DP, _DP, _DP,
                                    _DP, _DP, ctypes.c_int64, _DP, ctypes.c_int64,
                                    ctypes.POINTER(ctypes.c_int32), _DP]
        lib.dcpu_destroy.argtypes = [P]
        lib.dcpu_step.argtypes = [P, ctypes.c_int64]
        lib.dcpu_read_state.argtypes = [P, _DP, _DP, _DP, _DP]
        lib.dcpu_read_forces.argtypes = [P, _DP, _DP]
        lib.dcpu_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def threads() -> int:
    """OpenMP threads the baseline runs with (OMP_NUM_THREADS, else all cores)."""
    return int(_load().dcpu_threads())


def _f64(a, shape):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64).reshape(shape))


class CpuScene:
    """A scene advanced by the OpenMP CPU baseline.

    `elems` is an (m, 4) int32 array of vertex indices padded with -1 (point,
    segment, triangle or rectangle), `elem_radius` the element radii.
    """

    def __init__(self, params: dict, R, x, v, w, q, verts=None, elems=None, elem_radius=None):
        lib = _load()
        p = dcpu_params()
        for k in ("E", "nu", "rho", "e_n", "mu_s", "mu_r", "mu_t", "eta", "dt"):
            setattr(p, k, float(params[k]))
        p.g[:] = [float(c) for c in params.get("g", (0, 0, 0))]
        p.mesh_omega[:] = [float(c) for c in params.get("mesh_omega", (0, 0, 0))]
        p.mesh_center[:] = [float(c) for c in params.get("mesh_center", (0, 0, 0))]
        R = _f64(R, (-1,))
        n = R.shape[0]
        self.n = n
        x, v, w, q = _f64(x, (n, 3)), _f64(v, (n, 3)), _f64(w, (n, 3)), _f64(q, (n, 4))
        if elems is None or len(elems) == 0:
            V, El, Er, nv, ne = np.zeros(3), np.full(4, -1, np.int32), np.zeros(1), 0, 0
        else:
            V = _f64(verts, (-1, 3))
            El = np.ascontiguousarray(np.asarray(elems, dtype=np.int32).reshape(-1, 4))
            Er = _f64(np.zeros(len(El)) if elem_radius is None else elem_radius, (-1,))
            nv, ne = V.shape[0], El.shape[0]
        self._p = p
        self._lib = lib
        dp = lambda a: a.ctypes.data_as(_DP)  # noqa: E731
        self._h = lib.dcpu_create(ctypes.byref(p), n, dp(R), dp(x), dp(v), dp(w), dp(q), nv,
                                  dp(V), ne, El.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                  dp(Er))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._lib.dcpu_destroy(h)
            self._h = None

    def step(self, nsteps: int = 1) -> None:
        self._lib.dcpu_step(self._h, int(nsteps))

    def state(self) -> dict:
        n = self.n
        out = {k: np.empty((n, 3)) for k in ("x", "v", "w")}
        out["q"] = np.empty((n, 4))
        self._lib.dcpu_read_state(self._h, *(out[k].ctypes.data_as(_DP) for k in "xvwq"))
        return out

    def forces(self):
        F, T = np.empty((self.n, 3)), np.empty((self.n, 3))
        self._lib.dcpu_read_forces(self._h, F.ctypes.data_as(_DP), T.ctypes.data_as(_DP))
        return F, T


def cpu_model() -> str:
    """The host CPU's model name (or architecture), for the benchmark record."""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu model")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.machine() or "unknown"
