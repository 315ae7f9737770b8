"""Scene memory from the caller's allocator (dem_scene_create_with_allocator).

A scene whose every device buffer comes from PyTorch's caching allocator
runs bit for bit like one on cudaMalloc, its blocks count in torch's
statistics while it lives and go back to torch's pool when it is destroyed;
an allocator that runs dry or hands out a misaligned block makes creation
fail with DEM_ERR_NOMEM and gets every block back.
"""
import ctypes

import numpy as np
import pytest

from paper_2507_12610_gb300 import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_12610_gb300 import build
    build.build()
    from paper_2507_12610_gb300 import dem
    dem.load()
    return torch, dem


def run(dem, s, steps, **kw):
    sc = dem.Scene.from_dict(s, precision=dem.DEM_MIXED, **kw)
    sc.step(steps)
    assert sc.synchronize() == 0
    st = sc.state()
    return sc, st


def test_torch_allocator_runs_bitwise_alike_and_returns_its_memory(env):
    torch, dem = env
    s = scenes.drum_scene(n=20_000, seed=5, nn_dist=2.15e-3, speed=0.02)
    ref, a = run(dem, s, 300)
    ref.close()
    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    al = dem.TorchAllocator()
    sc, b = run(dem, s, 300, allocator=al)
    held = sum(al.live.values())
    assert len(al.live) > 10 and held > 0
    assert torch.cuda.memory_allocated() - m0 >= held  # torch rounds blocks up
    for k in ("x", "v", "w", "q"):
        assert np.array_equal(a[k], b[k]), k
    sc.close()
    assert not al.live
    assert torch.cuda.memory_allocated() == m0


def test_failing_allocator_reports_nomem_and_gets_every_block_back(env):
    torch, dem = env
    s = scenes.drum_scene(n=5_000, seed=5, nn_dist=2.15e-3, speed=0.02)

    class RunsDry(dem.TorchAllocator):
        def __init__(self, k):
            super().__init__()
            self.k = k

        def _alloc(self, nbytes, ctx):
            if len(self.live) >= self.k:
                return None
            return super()._alloc(nbytes, ctx)

    class Misaligned(dem.TorchAllocator):
        # every block starts 32 bytes into torch's block
        def __init__(self):
            super().__init__()
            self.base = {}

        def _alloc(self, nbytes, ctx):
            p = super()._alloc(nbytes + 32, ctx)
            self.base[p + 32] = p
            return p + 32

        def _free(self, ptr, ctx):
            super()._free(self.base.pop(ptr), ctx)

    torch.cuda.synchronize()
    m0 = torch.cuda.memory_allocated()
    for al in (RunsDry(5), Misaligned()):
        with pytest.raises(dem.DemError) as e:
            dem.Scene.from_dict(s, precision=dem.DEM_MIXED, allocator=al)
        assert e.value.code == dem.DEM_ERR_NOMEM
        assert not al.live
        assert torch.cuda.memory_allocated() == m0


def test_allocator_needs_both_functions(env):
    torch, dem = env
    s = scenes.lattice_box_scene((4, 4, 4), seed=3, walls=False)
    lib = dem.load()
    al = dem.TorchAllocator()
    sc = dem.Scene.from_dict(s, precision=dem.DEM_FP64)  # parameters and arrays as ctypes
    pp, h = sc._pp, ctypes.c_void_p()
    R = np.ascontiguousarray(s["R"], dtype=np.float64)
    x = np.ascontiguousarray(s["x"], dtype=np.float64)
    pa = dem.dem_particles(len(R), dem._p(R), dem._p(x), None, None, None)
    rc = lib.dem_scene_create_with_allocator(ctypes.byref(pp), ctypes.byref(pa),
                                             ctypes.byref(dem.dem_mesh()), None, al.alloc_fn,
                                             dem.FREE_FN(), None, ctypes.byref(h))
    assert rc == dem.DEM_ERR_INVALID and not h.value and not al.live
    sc.close()
