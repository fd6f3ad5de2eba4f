"""Converged CG stops on the true residual (Algorithm 1's stopping test taken
on b - A x, not on the recursive residual alone).

The recursive residual r_{j+1} = r_j - alpha A p_j drifts from b - A x_{j+1}
by rounding, the more so the worse the conditioning. On a mesh large and
ill-conditioned enough for that drift to show (lambda = 0, strong vertex
perturbation, 24^3 elements at N = 7), every CG form that reports HB_OK must
leave a true residual within the tolerance it was given:
  - the true residual is computed here on the whole vector with the GPU's FP64
    operator, whose rows are checked against the oracle's row-by-row
    evaluation at this size (1e-12 of the largest entry), so the bound holds
    under the oracle's A;
  - rel_res reports that true residual;
  - the stepwise form, which replaces no residual, reports the true residual
    at its recursive stop and says HB_ERR_NOT_CONVERGED when it is above rtol.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2202_12477_gb300 import hb, inputs  # noqa: E402

DIMS, N, RHO, LAM = (24, 24, 24), 7, 0.2, 0.0
RTOL = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


@pytest.fixture(scope="module")
def mesh():
    m = hb.Mesh(*DIMS, N, perturb=RHO, seed=0, fp32=True)
    yield m
    m.close()


def _true_rel(m, b, x):
    r = b - m.apply_A(x, lam=LAM)
    return float(torch.linalg.norm(r) / torch.linalg.norm(b))


def test_operator_rows_match_oracle_at_this_size(mesh):
    x = inputs.random_vector(mesh.n_global, seed=31)
    rows = inputs.sample_indices(mesh.n_global, 300, 32)
    ref = orc.apply_A_rows(DIMS, N, RHO, 0, x, rows, LAM)
    y = mesh.apply_A(torch.from_numpy(x).cuda(), lam=LAM).cpu().numpy()
    assert np.abs(y[rows] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("prec,precond", [(hb.HB_F64, 0), (hb.HB_F64, 1), (hb.HB_F64X, 0), (hb.HB_F64X, 1)])
def test_converged_cg_meets_tolerance_on_true_residual(mesh, prec, precond):
    b = mesh.rhs(kind=0, seed=0)
    x, res = mesh.cg(b, lam=LAM, rtol=RTOL, max_it=50000, prec=prec, precond=precond)
    assert res.status == hb.HB_OK, (res.status, res.rel_res, res.iters)
    rel = _true_rel(mesh, b, x)
    assert rel <= 1.01 * RTOL, rel
    assert abs(res.rel_res - rel) <= 1e-3 * rel, (res.rel_res, rel)


def test_stepwise_reports_true_residual(mesh):
    b = mesh.rhs(kind=0, seed=0)
    x = mesh.vec()
    mesh.cg_begin(b, x, lam=LAM, rtol=RTOL, max_it=50000)
    mesh.cg_iterate(50000)
    res = mesh.cg_finish()
    rel = _true_rel(mesh, b, x)
    assert abs(res.rel_res - rel) <= 1e-3 * rel, (res.rel_res, rel)
    assert res.status == (hb.HB_OK if rel <= RTOL else hb.HB_ERR_NOT_CONVERGED), (res.status, rel)


def test_partitioned_and_scattered_meet_tolerance_on_true_residual(mesh):
    b = mesh.rhs(kind=0, seed=0)
    part = hb.Part(mesh, 2, 2, 1)
    perm = torch.from_numpy(part.perm.astype(np.int64)).cuda()
    bp = b[perm].contiguous()
    xp, res = part.cg(bp, lam=LAM, rtol=RTOL, max_it=50000)
    assert res.status == hb.HB_OK, (res.status, res.rel_res)
    r = bp - part.apply_A(xp, lam=LAM)
    rel = float(torch.linalg.norm(r) / torch.linalg.norm(bp))
    assert rel <= 1.01 * RTOL and abs(res.rel_res - rel) <= 1e-3 * rel, (res.rel_res, rel)
    x = torch.empty_like(b)
    x[perm] = xp
    assert _true_rel(mesh, b, x) <= 1.01 * RTOL
    part.close()
    sc = hb.Scat(mesh)
    xl, res = sc.cg(sc.scatter(b), lam=LAM, rtol=RTOL, max_it=50000)
    assert res.status == hb.HB_OK, (res.status, res.rel_res)
    assert res.rel_res <= RTOL
    sc.close()
