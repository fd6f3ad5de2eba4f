"""Bounded device waits: a wait that can never complete gives up after about a
second, the kernel finishes, the failure comes back as HB_ERR_TIMEOUT and
the context stays usable. The waits are made to run out by a flag nothing
sets (an mbarrier no thread arrives at; a grid barrier that expects one block
more than were launched): no fault, no hang.
"""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2202_12477_gb300 import hb, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


@pytest.mark.parametrize("which", [0, 1], ids=["mbarrier", "grid_barrier"])
def test_wait_gives_up_and_reports(which):
    t0 = time.monotonic()
    assert hb.hb_selftest_wait(which) == hb.HB_ERR_TIMEOUT
    dt = time.monotonic() - t0
    assert 0.5 < dt < 30.0, dt
    # the context is still usable: an operator application keeps its parity
    m = hb.Mesh(3, 2, 2, 5, perturb=0.1, seed=1)
    o = orc.Mesh(3, 2, 2, 5, rho=0.1, seed=1)
    x = inputs.random_vector(m.n_global, seed=2)
    y = m.apply_A(torch.from_numpy(x).cuda(), lam=0.1).cpu().numpy()
    y_or = o.apply_A(x, 0.1, 0)
    assert np.linalg.norm(y - y_or) <= 1e-12 * np.linalg.norm(y_or)


def test_selftest_rejects_bad_argument():
    with pytest.raises(hb.HBError):
        hb.hb_selftest_wait(2)


def test_fused_cg_after_a_barrier_timeout():
    """The fused solver zeroes its barrier words at every launch: a solve
    after the self-test (and after another solve) is unaffected."""
    assert hb.hb_selftest_wait(1) == hb.HB_ERR_TIMEOUT
    m = hb.Mesh(4, 4, 4, 7, perturb=0.1, seed=0)
    o = orc.Mesh(4, 4, 4, 7, rho=0.1, seed=0)
    hb.lib().hb_set_cg_fused(m.handle, 2)
    b = m.rhs(kind=0, seed=0)
    x_or, _, _, _ = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=100)
    xs = []
    for _ in range(2):
        x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=100)
        assert res.status == hb.HB_OK and res.iters == 100
        assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-11 * np.linalg.norm(x_or)
        xs.append(x)
    assert torch.equal(xs[0], xs[1])
