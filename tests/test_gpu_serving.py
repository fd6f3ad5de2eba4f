"""The continuous-batching CG server, called through the C ABI.

Checks: every served solve meets its FP64 residual target under the oracle's
operator; a request gives bitwise the same solution alone and in a mix of
concurrent requests (fixed grids and per-slot reductions); requests queue
when slots or memory run out; a request that can never fit is refused.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2202_12477_gb300 import hb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


def _ng(ex, ey, ez, N):
    return (N * ex - 1) * (N * ey - 1) * (N * ez - 1)


REQ = dict(ex=3, ey=2, ez=3, N=5, perturb=0.15, seed=4, rhs_seed=7, lam=0.1, rtol=1e-10)


def _check_residual(req, x):
    o = orc.Mesh(req["ex"], req["ey"], req["ez"], req["N"], rho=req["perturb"], seed=req["seed"])
    b = o.rhs(kind=0, seed=req["rhs_seed"])
    r = b - o.apply_A(x, req["lam"])
    return np.linalg.norm(r) / np.linalg.norm(b)


def test_served_solve_meets_fp64_residual():
    srv = hb.Server(8 << 30, max_slots=4, iters_per_launch=8)
    t = srv.submit(**REQ, keep_x=True)
    res, x = srv.wait(t, _ng(REQ["ex"], REQ["ey"], REQ["ez"], REQ["N"]))
    assert res.status == hb.HB_OK and res.rel_res <= 1e-10
    assert _check_residual(REQ, x) <= 1.01e-10
    assert res.outer_iters >= 1 and res.iters > 0
    srv.close()


def test_same_result_alone_and_in_a_mix():
    ng = _ng(REQ["ex"], REQ["ey"], REQ["ez"], REQ["N"])
    srv = hb.Server(8 << 30, max_slots=8, iters_per_launch=8)
    t = srv.submit(**REQ, keep_x=True)
    _, x_alone = srv.wait(t, ng)
    # the same request among others of different sizes, degrees and tolerances
    others = [dict(ex=2, ey=2, ez=2, N=3, rtol=1e-8), dict(ex=4, ey=3, ez=2, N=7, rtol=1e-10),
              dict(ex=2, ey=3, ez=2, N=9, rtol=1e-8), dict(ex=5, ey=5, ez=4, N=3, rtol=1e-10),
              dict(ex=2, ey=2, ez=3, N=11, rtol=1e-8)]
    tickets = [srv.submit(**o, keep_x=True) for o in others[:3]]
    t2 = srv.submit(**REQ, keep_x=True)
    tickets += [srv.submit(**o, keep_x=True) for o in others[3:]]
    _, x_mix = srv.wait(t2, ng)
    assert np.array_equal(x_alone, x_mix)
    for o, tk in zip(others, tickets):
        res, x = srv.wait(tk, _ng(o["ex"], o["ey"], o["ez"], o["N"]))
        assert res.status == hb.HB_OK, (o, res.status)
        full = dict(perturb=0.1, seed=0, rhs_seed=0, lam=0.1)
        full.update(o)
        assert _check_residual(full, x) <= 1.01 * o["rtol"]
    st = srv.stats()
    assert st.completed == 2 + len(others) and st.active == 0 and st.pending == 0
    # the worker's time by phase: building requests, rounds, retiring
    assert st.rounds > 0 and st.admit_s > 0.0 and st.round_s > 0.0 and st.retire_s >= 0.0
    srv.close()


def test_queueing_when_slots_and_memory_are_short():
    # one slot: requests wait for each other and all finish
    srv = hb.Server(8 << 30, max_slots=1, iters_per_launch=4)
    ts = [srv.submit(ex=2, ey=2, ez=2, N=n, rtol=1e-8) for n in (3, 4, 5)]
    for t in ts:
        res, _ = srv.wait(t)
        assert res.status == hb.HB_OK
    assert srv.stats().rounds > 0
    srv.close()
    # a request that can never fit the budget is refused, the next still runs
    srv = hb.Server(64 << 20, max_slots=4, iters_per_launch=4)
    big = srv.submit(ex=32, ey=32, ez=32, N=11, rtol=1e-8)
    small = srv.submit(ex=2, ey=2, ez=2, N=3, rtol=1e-8)
    res, _ = srv.wait(big)
    assert res.status == hb.HB_ERR_NOMEM
    res, _ = srv.wait(small)
    assert res.status == hb.HB_OK
    srv.close()


def test_server_argument_errors():
    srv = hb.Server(1 << 30, max_slots=2, iters_per_launch=2)
    with pytest.raises(hb.HBError):
        srv.submit(ex=2, ey=2, ez=2, N=12)
    with pytest.raises(hb.HBError):
        srv.submit(ex=2, ey=2, ez=2, N=3, rtol=0.0)
    with pytest.raises(hb.HBError):
        srv.poll(999)  # never issued
    srv.close()


def test_failed_round_resolves_every_ticket_and_frees_memory():
    # The failure is made on the host (the test hook makes the worker treat a
    # round as a failed launch); no device work faults.
    srv = hb.Server(8 << 30, max_slots=2, iters_per_launch=2)
    reqs = [dict(ex=6, ey=6, ez=6, N=7, rtol=1e-12, seed=s, rhs_seed=s) for s in range(5)]
    tickets = [srv.submit(**r) for r in reqs]
    srv.inject_round_error()
    statuses = [srv.wait(t, timeout=120.0)[0].status for t in tickets]
    assert all(s in (hb.HB_OK, hb.HB_ERR_CUDA) for s in statuses), statuses
    assert hb.HB_ERR_CUDA in statuses
    # a request that was being built when the round failed releases its
    # memory once its build ends
    import time
    t0 = time.time()
    st = srv.stats()
    while (st.active or st.mem_used) and time.time() - t0 < 30.0:
        time.sleep(0.01)
        st = srv.stats()
    assert st.active == 0 and st.pending == 0 and st.mem_used == 0
    with pytest.raises(hb.HBError):
        srv.submit(**REQ)  # a stopped server takes no new work
    srv.close()
