"""Host-side helpers of bench.py (no GPU): the workload shapes the bench line
is quoted on and the serving stream it replays.

Checks:
- the degree-sweep box holds about 1.28e8 local nodes at every degree,
  with Ex = Ey a multiple of 8;
- the serving stream is seeded (the same requests every run) and stays inside
  its stated ranges (Ek 2..32, N odd in 3..11, rtol 1e-8 or 1e-10);
- the failure summary counts statuses by name and keeps the first message.
"""
import bench
from paper_2202_12477_gb300 import hb


def test_degree_sweep_box_sizes():
    for N in range(1, 16):
        ex, ey, ez = bench.c2_dims(N)
        n = N + 1
        nl = ex * ey * ez * n ** 3
        assert ex == ey and ex % 8 == 0 and ez >= 1
        assert 0.85e8 <= nl <= 1.29e8, (N, ex, ez, nl)
    # the headline box at N = 7
    assert bench.c2_dims(7) == (64, 64, 61)


def test_serving_stream_is_seeded_and_in_range():
    a = bench._c5_requests(300, 2, 32)
    b = bench._c5_requests(300, 2, 32)
    assert a == b
    assert len(a) == 300
    for r in a:
        assert 2 <= r["ex"] <= 32 and r["ex"] == r["ey"] == r["ez"]
        assert r["N"] in (3, 5, 7, 9, 11)
        assert r["rtol"] in (1e-8, 1e-10)
    # both tolerances and every degree occur in the first 300
    assert {r["N"] for r in a} == {3, 5, 7, 9, 11}
    assert {r["rtol"] for r in a} == {1e-8, 1e-10}


def test_failure_summary():
    bench._FAIL_MSG.clear()
    bench._FAIL_MSG["HB_ERR_CUDA"] = "round: unspecified launch failure"
    out = bench._not_ok([hb.HB_OK, hb.HB_ERR_CUDA, hb.HB_OK, hb.HB_ERR_CUDA, hb.HB_ERR_NOMEM])
    assert out["HB_ERR_CUDA"] == {"count": 2, "message": "round: unspecified launch failure"}
    assert out["HB_ERR_NOMEM"] == {"count": 1, "message": ""}
    assert "HB_OK" not in out
    assert bench._not_ok([hb.HB_OK] * 3) == {}
    bench._FAIL_MSG.clear()
