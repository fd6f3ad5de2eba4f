"""Tensor-core operand layouts (tcgen05.mma kind::f16 with FP16 operands in
shared memory and an FP32 accumulator in tensor memory), checked through the
C ABI against numpy: D = A B^T on integer-valued inputs small enough that
every product and every sum is exact in FP32, so the comparison is bit-exact.
These are the layouts the tensor-core element kernel stages its operands in:
K-major A and B (the entry point can also stage A MN-major, a layout the
kernel does not use)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2202_12477_gb300 import hb  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


def test_tc_layouts_exact():
    mode = 0  # K-major A and B, the layouts the element kernel stages
    rng = np.random.Generator(np.random.PCG64(5))
    A = rng.integers(-256, 257, size=(128, 48)).astype(np.float32)
    B = rng.integers(-256, 257, size=(48, 48)).astype(np.float32)
    D, st = hb.hb_tc_selftest(mode, A, B)
    assert st == hb.HB_OK
    want = A.astype(np.float64) @ B.astype(np.float64).T
    assert np.abs(want).max() < 2 ** 24
    assert np.array_equal(D.astype(np.float64), want)


# ---------------------------------------------------------------- the tensor-core FP64 element kernel

from oracle import oracle as orc  # noqa: E402
from paper_2202_12477_gb300 import inputs  # noqa: E402

TC = hb.HB_VARIANT_TC
TC_VARIANTS = hb.VARIANTS_TC


def _pair(dims, rho=0.15, seed=0, faces=0x3F, variant=TC):
    m = hb.Mesh(*dims, 7, perturb=rho, seed=seed, faces=faces, fp32=False)
    o = orc.Mesh(*dims, 7, rho=rho, seed=seed, faces=faces)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
    return m, o


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _check(y, y_or, bar=1e-12):
    s = np.abs(y_or).max()  # compare at unit scale (the norms of 1e200-sized vectors overflow)
    assert np.linalg.norm((y - y_or) / s) <= bar * np.linalg.norm(y_or / s)
    assert np.abs(y - y_or).max() <= bar * s


# one element, one whole tile, ragged last tiles, several tiles per block
@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (3, 1, 1), (3, 3, 3), (5, 4, 3)])
@pytest.mark.parametrize("screen,lam", [(0, 0.1), (1, 0.7), (0, 0.0)])
@pytest.mark.parametrize("faces", [0x3F, 0x15, 0x00])
@pytest.mark.parametrize("variant", TC_VARIANTS)
def test_tc_apply_matches_oracle(dims, screen, lam, faces, variant):
    m, o = _pair(dims, seed=sum(dims) + faces, faces=faces, variant=variant)
    x = inputs.random_vector(m.n_global, seed=400 + sum(dims))
    y = m.apply_A(_dev(x), lam=lam, screen=screen).cpu().numpy()
    _check(y, o.apply_A(x, lam, screen))
    m.close()


@pytest.mark.parametrize("scale", [1e-200, 1e-30, 1.0, 1e30, 1e200])
@pytest.mark.parametrize("variant", TC_VARIANTS)
def test_tc_apply_any_magnitude(scale, variant):
    """The fixed-point grid follows each element's largest exponent: results
    keep the FP64 bar at any scale, and across elements of very different
    magnitudes (each element's rounding is relative to its own values)."""
    m, o = _pair((3, 3, 2), seed=3, variant=variant)
    x = inputs.random_vector(m.n_global, seed=41) * scale
    y = m.apply_A(_dev(x), lam=0.1).cpu().numpy()
    _check(y, o.apply_A(x, 0.1, 0))
    # magnitudes spread over 60 decades between DOFs
    w = 10.0 ** inputs.random_vector(m.n_global, seed=42, kind="uniform") * 30.0
    xw = x / scale * w
    y = m.apply_A(_dev(xw), lam=0.1).cpu().numpy()
    _check(y, o.apply_A(xw, 0.1, 0))
    m.close()


def test_tc_zero_and_nonfinite():
    m, o = _pair((3, 2, 2), seed=5)
    z = torch.zeros(m.n_global, dtype=torch.float64, device="cuda")
    assert torch.count_nonzero(m.apply_A(z, lam=0.1)).item() == 0
    # a NaN in x: NaN wherever the FP64 pencil kernel gives NaN, and only at
    # DOFs of the elements that hold the NaN; elsewhere the oracle's values
    x = inputs.random_vector(m.n_global, seed=43)
    g_bad = m.n_global // 2
    x[g_bad] = np.nan
    y_tc = m.apply_A(_dev(x), lam=0.1).cpu().numpy()
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 3)
    y_ref = m.apply_A(_dev(x), lam=0.1).cpu().numpy()
    assert np.isnan(y_tc[np.isnan(y_ref)]).all()
    l2g = m.l2g().reshape(m.E, -1)
    touched = np.unique(l2g[(l2g == g_bad).any(axis=1)])
    touched = touched[touched >= 0]
    assert not np.isnan(np.delete(y_tc, touched)).any()
    far = np.setdiff1d(np.arange(m.n_global), touched)
    x0 = x.copy()
    x0[g_bad] = 0.0
    y_or = o.apply_A(x0, 0.1, 0)
    assert np.abs(y_tc[far] - y_or[far]).max() <= 1e-12 * np.abs(y_or).max()
    m.close()


def test_tc_variant_rules():
    m = hb.Mesh(2, 2, 2, 5, fp32=True)
    with pytest.raises(hb.HBError):
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, TC)  # built for N = 7 only
    m.close()
    m = hb.Mesh(2, 2, 2, 7, fp32=True)
    for prec in (hb.HB_F32, hb.HB_F64X):
        with pytest.raises(hb.HBError):
            hb.hb_set_kernel_variant(m.handle, prec, TC)
    v, ms = hb.hb_autotune(m.handle, hb.HB_F64, reps=2)
    assert all(t in ms for t in TC_VARIANTS) and v in ms
    m.close()


@pytest.mark.parametrize("variant", TC_VARIANTS)
def test_tc_cg_follows_oracle(variant):
    """Config 1 (4x4x4, N = 7): 100 fixed FP64 CG iterations with the
    tensor-core kernel in the launched solver, against the oracle's iterate;
    then a converged solve whose true residual meets the tolerance."""
    m, o = _pair((4, 4, 4), rho=0.1, seed=0, variant=variant)
    hb.lib().hb_set_cg_fused(m.handle, 1)
    b = m.rhs(kind=0, seed=0)
    x_or, *_ = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=100)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=100)
    assert res.status == hb.HB_OK and res.iters == 100
    assert np.linalg.norm(x.cpu().numpy() - x_or) <= 1e-12 * np.linalg.norm(x_or)
    x2, r2 = m.cg(b, lam=0.1, rtol=1e-11, max_it=5000)
    assert r2.status == hb.HB_OK
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - o.apply_A(x2.cpu().numpy(), 0.1)) <= 1.01e-11 * np.linalg.norm(bn)
    m.close()


@pytest.mark.parametrize("variant", TC_VARIANTS)
def test_tc_full_size_sampled_rows(variant):
    """The degree-sweep box at N = 7 (64 x 64 x 61, 1.28e8 local nodes), in
    the launch configuration the benchmark times: sampled rows against the
    oracle's row-by-row evaluation, and symmetry on the whole vector."""
    dims = (64, 64, 61)
    m = hb.Mesh(*dims, 7, perturb=0.1, seed=0, fp32=False)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
    x = inputs.random_vector(m.n_global, seed=11)
    rows = inputs.sample_indices(m.n_global, 600, 12)
    ref = orc.apply_A_rows(dims, 7, 0.1, 0, x, rows, 0.1)
    xd = _dev(x)
    y = m.apply_A(xd, lam=0.1).cpu().numpy()
    assert np.abs(y[rows] - ref).max() <= 1e-12 * np.abs(ref).max()
    z = _dev(inputs.random_vector(m.n_global, seed=13))
    a = m.dot(xd, m.apply_A(z, lam=0.1))
    b = m.dot(z, m.apply_A(xd, lam=0.1))
    assert abs(a - b) <= 1e-12 * abs(a)
    m.close()
