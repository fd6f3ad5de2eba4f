"""Scattered (NekBone) storage against the oracle and the assembled path.

x_L = Z x_G; the operator b_L = (Z Z^T S_L + lambda I) x_L must equal
Z (A x_G) (the oracle's result at every copy, 0 at masked nodes); weighted
inner products equal the assembled ones; CG on scattered vectors follows the
oracle's iterates (its solution is Z x_oracle).
"""
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


def _setup(dims, N, rho=0.15, seed=0, faces=0x3F):
    m = hb.Mesh(*dims, N, perturb=rho, seed=seed, faces=faces, fp32=False)
    o = orc.Mesh(*dims, N, rho=rho, seed=seed, faces=faces)
    sc = hb.Scat(m)
    l2g = o.l2g().reshape(-1).astype(np.int64)
    return m, o, sc, l2g


def _Z(xG, l2g):
    return np.where(l2g >= 0, xG[np.maximum(l2g, 0)], 0.0)


CASES = [((2, 2, 2), 1), ((3, 2, 2), 3), ((3, 3, 3), 5), ((3, 3, 2), 7), ((2, 2, 1), 10), ((1, 2, 2), 15)]


@pytest.mark.parametrize("dims,N", CASES)
def test_scatter_and_weights(dims, N):
    m, o, sc, l2g = _setup(dims, N, seed=N)
    xG = inputs.random_vector(m.n_global, seed=N)
    xL = sc.scatter(torch.from_numpy(xG).cuda()).cpu().numpy()
    assert np.array_equal(xL, _Z(xG, l2g))
    # weights through the weighted dot: (1_L, 1_L)_c = number of DOFs, (Zx, Zy)_c = x.y
    one = sc.scatter(torch.ones(m.n_global, dtype=torch.float64, device="cuda"))
    assert sc.dot(one, one) == float(m.n_global)
    yG = inputs.random_vector(m.n_global, seed=N + 100)
    yL = sc.scatter(torch.from_numpy(yG).cuda())
    exact = float(np.dot(xG, yG))
    assert abs(sc.dot(torch.from_numpy(xL).cuda(), yL) - exact) <= 1e-14 * np.abs(xG * yG).sum()


@pytest.mark.parametrize("dims,N", CASES)
@pytest.mark.parametrize("screen,lam", [(0, 0.1), (1, 0.7), (0, 0.0)])
def test_scattered_apply_matches_oracle(dims, N, screen, lam):
    m, o, sc, l2g = _setup(dims, N, seed=N + 1)
    xG = inputs.random_vector(m.n_global, seed=200 + N)
    want = _Z(o.apply_A(xG, lam, screen), l2g)
    xL = sc.scatter(torch.from_numpy(xG).cuda())
    y = sc.apply_A(xL, lam=lam, screen=screen).cpu().numpy()
    assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()
    assert np.all(y[l2g < 0] == 0.0)
    # every copy of a DOF holds the same value
    yG = np.zeros(m.n_global)
    yG[l2g[l2g >= 0]] = y[l2g >= 0]
    assert np.array_equal(_Z(yG, l2g), y)


def test_scattered_apply_neumann_and_partial_faces():
    for faces in (0x00, 0x2A):
        m, o, sc, l2g = _setup((3, 2, 2), 4, seed=3, faces=faces)
        xG = inputs.random_vector(m.n_global, seed=9)
        want = _Z(o.apply_A(xG, 0.3, 0), l2g)
        y = sc.apply_A(sc.scatter(torch.from_numpy(xG).cuda()), lam=0.3).cpu().numpy()
        assert np.abs(y - want).max() <= 1e-12 * np.abs(want).max()


def test_scattered_cg_follows_oracle():
    m, o, sc, l2g = _setup((3, 3, 3), 5, seed=4)
    bG = m.rhs(kind=0, seed=4)
    x_or, it_or, rel_or, st_or = o.cg(bG.cpu().numpy(), 0.1, rtol=0.0, max_it=50)
    bL = sc.scatter(bG)
    xL, res = sc.cg(bL, lam=0.1, rtol=0.0, max_it=50)
    assert res.status == hb.HB_OK and res.iters == 50
    want = _Z(x_or, l2g)
    assert np.linalg.norm(xL.cpu().numpy() - want) <= 1e-9 * np.linalg.norm(want)
    x2, res2 = sc.cg(bL, lam=0.1, rtol=1e-10, max_it=5000)
    assert res2.status == hb.HB_OK and res2.rel_res <= 1e-10
    # the assembled solver reaches the same solution
    xa, ra = m.cg(bG, lam=0.1, rtol=1e-10, max_it=5000)
    want = _Z(xa.cpu().numpy(), l2g)
    assert np.linalg.norm(x2.cpu().numpy() - want) <= 1e-8 * np.linalg.norm(want)
    assert abs(res2.iters - ra.iters) <= 2


def test_scat_invalid_arguments():
    m, o, sc, l2g = _setup((2, 2, 2), 3)
    x = sc.vec()
    st = hb.lib().hb_scat_apply_A(sc.handle, 0, 0.1, hb.C.c_void_p(x.data_ptr()), hb.C.c_void_p(x.data_ptr()),
                                  hb._stream_ptr(None))
    assert st == hb.HB_ERR_ARG
    st = hb.lib().hb_scat_apply_A(sc.handle, 7, 0.1, hb.C.c_void_p(x.data_ptr()), hb.C.c_void_p(sc.vec().data_ptr()),
                                  hb._stream_ptr(None))
    assert st == hb.HB_ERR_ARG
