"""Parity at the benchmark's full sizes (about 1.28e8 local nodes), in the
launch configuration bench.py times.

The full oracle cannot hold these meshes, so (a) sampled rows of A x are
compared one by one with the oracle's row-by-row evaluation, and (b)
properties that hold at any size are checked on the whole vector: symmetry
x.Ay = y.Ax, and after CG iterations the recursive residual against the true
residual b - A x.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from oracle import oracle as orc  # noqa: E402
from paper_2202_12477_gb300 import hb, inputs  # noqa: E402

# degree-sweep configuration: elements per axis for ~1.28e8 local nodes
FULL = {7: (64, 64, 61), 15: (32, 32, 30)}


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


def _rows(m, dims, N, count, seed):
    """Seeded sample plus structured rows: first, last, and DOFs on element
    vertices, edges, faces and interiors near the middle of the box."""
    rows = set(inputs.sample_indices(m.n_global, count, seed).tolist())
    NXu, NYu = N * dims[0] - 1, N * dims[1] - 1
    I0, J0, K0 = N * (dims[0] // 2), N * (dims[1] // 2), N * (dims[2] // 2)
    for di, dj, dk in [(0, 0, 0), (1, 0, 0), (1, 1, 0), (1, 1, 1), (0, 1, 1), (N // 2, N // 2, N // 2)]:
        I, J, K = I0 + di, J0 + dj, K0 + dk
        rows.add((I - 1) + NXu * ((J - 1) + NYu * (K - 1)))
    return np.array(sorted(rows), dtype=np.int64)


@pytest.mark.parametrize("N", [7, 15])
def test_full_size_apply_sampled_rows(N):
    dims = FULL[N]
    m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=True)
    assert m.n_local == dims[0] * dims[1] * dims[2] * (N + 1) ** 3
    x = inputs.random_vector(m.n_global, seed=11)
    xd = torch.from_numpy(x).cuda()
    rows = _rows(m, dims, N, 600, seed=12)
    ref = orc.apply_A_rows(dims, N, 0.1, 0, x, rows, 0.1)
    scale = np.abs(ref).max()
    for variant in hb.VARIANTS:
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
        y = m.apply_A(xd, lam=0.1).cpu().numpy()
        err = np.abs(y[rows] - ref).max()
        assert err <= 1e-12 * scale, (variant, err / scale)
    # double-float element kernel on the same FP64 data
    for variant in hb.VARIANTS_F64X:
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64X, variant)
        y = m.apply_A(xd, lam=0.1, prec=hb.HB_F64X).cpu().numpy()
        err = np.abs(y[rows] - ref).max()
        assert err <= 1e-12 * scale, ("f64x", variant, err / scale)
    # FP32 operator (the mixed-precision inner product) on the same rows
    x32 = x.astype(np.float32)
    ref32 = orc.apply_A_rows(dims, N, 0.1, 0, x32.astype(np.float64), rows, 0.1)
    x32d = torch.from_numpy(x32).cuda()
    for variant in (3, 35, 131):  # plain, warp-specialised staged, lattice gather
        hb.hb_set_kernel_variant(m.handle, hb.HB_F32, variant)
        y32 = m.apply_A(x32d, lam=0.1).cpu().numpy().astype(np.float64)
        assert np.linalg.norm(y32[rows] - ref32) <= 2e-5 * np.linalg.norm(ref32), variant
    # symmetry on the whole vector
    z = torch.from_numpy(inputs.random_vector(m.n_global, seed=13)).cuda()
    a = m.dot(xd, m.apply_A(z, lam=0.1))
    b = m.dot(z, m.apply_A(xd, lam=0.1))
    assert abs(a - b) <= 1e-12 * abs(a)
    m.close()


def test_full_size_cg_residual_identity():
    """Bench configuration: after 5 FP64 CG iterations the recursive residual
    equals the true residual b - A x (computed with the parity-checked A)."""
    N, dims = 7, FULL[7]
    m = hb.Mesh(*dims, N, perturb=0.1, seed=0, fp32=False)
    b = m.rhs(kind=0, seed=0)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=5)
    assert res.iters == 5 and res.status == hb.HB_OK
    r = b - m.apply_A(x, lam=0.1)
    true_rel = float(torch.linalg.norm(r) / torch.linalg.norm(b))
    assert abs(true_rel - res.rel_res) <= 1e-10 * res.rel_res + 1e-14
    # the uniform rhs equals the oracle's generator on sampled DOFs
    rows = inputs.sample_indices(m.n_global, 200, 3)
    bh = b.cpu().numpy()[rows]
    NXu, NYu = N * dims[0] - 1, N * dims[1] - 1
    NX, NY = N * dims[0] + 1, N * dims[1] + 1
    for g, v in zip(rows.tolist(), bh.tolist()):
        I, J, K = g % NXu + 1, (g // NXu) % NYu + 1, g // (NXu * NYu) + 1
        assert v == 2.0 * orc.u01(0, 2, I + NX * (J + NY * K)) - 1.0
    m.close()
