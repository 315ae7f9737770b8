"""The C-ABI library builds, loads and exports every symbol include/dem.h declares.

Runs without a GPU: it only compiles the library, loads it and looks up the
exported names (no CUDA call is made).
"""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "dem.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dem_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2507_12610_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("dem_scene_create", "dem_step", "dem_read_state", "dem_scene_destroy"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_names_match_header():
    from paper_2507_12610_gb300 import dem
    assert sorted(dem.EXPORTS) == declared_functions()


def test_status_strings_without_gpu(lib):
    lib.dem_status_string.restype = ctypes.c_char_p
    assert lib.dem_status_string(0) == b"ok"
    assert lib.dem_status_string(2) == b"list capacity exceeded"


def test_struct_layouts_match_header():
    # sizes of the ctypes mirrors against the C layout (all fields naturally aligned)
    from paper_2507_12610_gb300 import dem
    assert ctypes.sizeof(dem.dem_params) == (8 * (8 + 3 + 1 + 3 + 3 + 1 + 3 + 3) + 4 * 4
                                             + 8 + 8 * (3 + 3 + 2 + 3 + 3) + 4 + 4 + 8 + 4 + 4)
    assert ctypes.sizeof(dem.dem_particles) == 8 * 6 + 8 + 8 + 8
    assert ctypes.sizeof(dem.dem_mesh) == 8 * 8
    assert ctypes.sizeof(dem.dem_stats) == 8 * 6 + 4 * 4 + 8 * 2


def test_oracle_and_library_share_no_code():
    # the oracle must not include, import or link anything of the CUDA path and
    # vice versa
    osrc = open(os.path.join(ROOT, "oracle", "dem_oracle.cpp")).read()
    assert "dem.h" not in osrc and "paper_2507_12610_gb300" not in osrc
    opy = open(os.path.join(ROOT, "oracle", "oracle.py")).read()
    assert "paper_2507_12610_gb300" not in opy
    csrc = os.path.join(ROOT, "paper_2507_12610_gb300", "csrc")
    for f in os.listdir(csrc):
        assert "oracle" not in open(os.path.join(csrc, f)).read().lower(), f
    for f in ("dem.py", "build.py", "scenes.py"):
        txt = open(os.path.join(ROOT, "paper_2507_12610_gb300", f)).read()
        assert "import oracle" not in txt and "from oracle" not in txt, f


def test_bad_mesh_elements_are_rejected_on_the_host():
    # element checks run before any CUDA call, so this needs no GPU: a
    # rectangle without right angles, a pad other than -1, a vertex index out
    # of range, an empty row and a negative radius each give DEM_ERR_INVALID
    import numpy as np
    from paper_2507_12610_gb300 import build, dem, scenes
    build.build()
    s = scenes.primitives_scene(n_side=(2, 2, 2))
    E, er = s["elems"], s["elem_radius"]
    V = s["verts"]
    skew = V.copy()
    skew[E[6, 2]] += np.array([0.0, 1e-4, 0.0])  # corner c off the plate's plane
    cases = []
    e = E.copy(); e[7, 3] = 0; cases.append((V, e, er))       # pad not -1
    e = E.copy(); e[8, 0] = len(V); cases.append((V, e, er))  # index out of range
    e = E.copy(); e[8, :] = -1; cases.append((V, e, er))      # no vertex
    r = er.copy(); r[7] = -1e-3; cases.append((V, E, r))      # negative radius
    cases.append((skew, E, er))                               # not a rectangle
    for Vc, Ec, rc in cases:
        bad = dict(s, verts=Vc, elems=Ec, elem_radius=rc)
        with pytest.raises(dem.DemError) as err:
            dem.Scene.from_dict(bad)
        assert err.value.code == dem.DEM_ERR_INVALID
