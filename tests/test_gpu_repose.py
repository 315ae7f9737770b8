"""The piling example (Sec. 5) at a small size: a spawned stream between two
plates forms a heap with straight flanks; both precisions agree on its angle
of repose and packing (the full-size statistics are a longer run)."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def repose():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2507_12610_gb300 import build
    build.build()
    from paper_2507_12610_gb300 import repose as r
    return r


def test_small_heap_in_both_precisions(repose):
    out = {p: repose.run(n=3000, precision=p, max_time=3.0) for p in (0, 1)}
    for r in out.values():
        assert r["status"] == 0 and r["settled"] and r["active"] == 3000
        # a small heap: flanks well below the large-heap angle, both alike
        assert 20.0 < r["theta"] < 45.0
        assert abs(r["theta_left"] - r["theta_right"]) < 6.0
        assert 0.42 < r["packing_core"] < 0.62
    # 3000 grains: one realisation each, a few per cent apart at most
    assert abs(out[0]["theta"] - out[1]["theta"]) < 0.06 * out[0]["theta"]
    assert abs(out[0]["packing_core"] - out[1]["packing_core"]) < 0.03
