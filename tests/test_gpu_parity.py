"""GPU parity: the CUDA library, called through its C ABI, against the FP64
oracle on the same seeded inputs.

Bars (from the arithmetic; see the design notes):
  - node map and DOF counts: bit-exact;
  - geometric factors: 1e-13 of the largest factor (two routes to the Jacobian);
  - FP64 A x: ||y - y_oracle||_2 <= 1e-12 ||y_oracle||_2 and
    max |y - y_oracle| <= 1e-12 max |y_oracle| (a few units of rounding times the
    ~6(N+1) terms of each contraction and the summation over copies);
  - FP32 A x: 2e-5 relative (FP32 rounding, 2^-24, times the same term counts);
  - dot: 1e-14 relative to the correctly rounded sum (math.fsum);
  - CG, fixed 100 iterations: 1e-12 relative to the oracle's iterate;
  - converged CG: both reach rtol and agree to 10 rtol.
"""
import math

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


def _pair(dims, N, rho=0.1, seed=0, faces=0x3F):
    m = hb.Mesh(*dims, N, perturb=rho, seed=seed, faces=faces, fp32=True)
    o = orc.Mesh(*dims, N, rho=rho, seed=seed, faces=faces)
    return m, o


def _to_dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ---------------------------------------------------------------- mesh

@pytest.mark.parametrize("dims,N,faces", [((2, 3, 2), 3, 0x3F), ((3, 2, 2), 2, 0x00), ((2, 2, 3), 4, 0x15),
                                          ((1, 1, 1), 1, 0x3F), ((5, 5, 5), 7, 0x3F), ((2, 2, 2), 15, 0x2A)])
def test_node_map_bit_exact(dims, N, faces):
    m, o = _pair(dims, N, faces=faces)
    assert m.n_global == o.n_global
    np.testing.assert_array_equal(m.l2g(), o.l2g().ravel())


@pytest.mark.parametrize("N,Ex,Ey,Ez,NG", [(7, 50, 50, 50, 42508549), (15, 24, 24, 24, 46268279),
                                           (7, 5, 10, 15, 243984), (15, 2, 2, 6, 74849)])
def test_dof_counts_of_paper_meshes(N, Ex, Ey, Ez, NG):
    m = hb.Mesh(Ex, Ey, Ez, N, fp32=False)
    assert m.n_global == NG
    m.close()


@pytest.mark.parametrize("dims,N,rho", [((2, 3, 2), 1, 0.2), ((3, 2, 2), 4, 0.3), ((2, 2, 2), 7, 0.1),
                                        ((2, 1, 2), 12, 0.25), ((1, 2, 1), 15, 0.1)])
def test_geometric_factors(dims, N, rho):
    m, o = _pair(dims, N, rho=rho, seed=7)
    n = N + 1
    geo = m.geo().reshape(m.E, n, 7, n, n)          # [e][k][c][j][i]
    G, Jw = o.geo()                                  # [e][k][j][i][6], [e][k][j][i]
    ref = np.concatenate([np.moveaxis(G, -1, 2), Jw[:, :, None]], axis=2)  # [e][k][c][j][i]
    # the off-diagonal entries are sums of products of the same Jacobian-inverse
    # entries as the diagonal ones: their rounding scales with the whole tensor
    gscale = np.abs(ref[:, :, :6]).max()
    for c in range(6):
        assert np.abs(geo[:, :, c] - ref[:, :, c]).max() <= 1e-13 * gscale, c
    assert np.abs(geo[:, :, 6] - ref[:, :, 6]).max() <= 1e-13 * np.abs(ref[:, :, 6]).max()
    assert abs(m.info.min_detJ - o.min_detJ) <= 1e-13 * o.min_detJ


# ---------------------------------------------------------------- operator

OP_CASES = [((2, 2, 2), 1), ((5, 3, 2), 2), ((3, 3, 3), 3), ((4, 3, 3), 4), ((3, 2, 3), 5), ((3, 3, 2), 6),
            ((3, 3, 3), 7), ((2, 3, 2), 8), ((2, 2, 3), 9), ((2, 2, 2), 10), ((3, 1, 2), 11), ((2, 2, 1), 12),
            ((1, 2, 2), 13), ((2, 1, 1), 14), ((1, 2, 2), 15)]


@pytest.mark.parametrize("dims,N", OP_CASES)
@pytest.mark.parametrize("screen,lam", [(0, 0.1), (1, 0.7), (0, 0.0)])
def test_apply_A_fp64(dims, N, screen, lam):
    m, o = _pair(dims, N, rho=0.15, seed=N)
    x = inputs.random_vector(m.n_global, seed=100 + N)
    y_or = o.apply_A(x, lam, screen)
    y = m.apply_A(_to_dev(x), lam=lam, screen=screen).cpu().numpy()
    assert _rel(y, y_or) <= 1e-12
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()


@pytest.mark.parametrize("variant", hb.VARIANTS)
@pytest.mark.parametrize("dims,N", OP_CASES)
def test_apply_A_fp64_every_variant(dims, N, variant):
    m, o = _pair(dims, N, rho=0.2, seed=N + 1)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F32, variant)
    x = inputs.random_vector(m.n_global, seed=300 + N)
    y_or = o.apply_A(x, 0.1, 0)
    y = m.apply_A(_to_dev(x), lam=0.1).cpu().numpy()
    assert _rel(y, y_or) <= 1e-12
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()
    x32 = x.astype(np.float32)
    y32_or = o.apply_A(x32.astype(np.float64), 0.1, 0)
    y32 = m.apply_A(_to_dev(x32, torch.float32), lam=0.1).cpu().numpy().astype(np.float64)
    assert _rel(y32, y32_or) <= 2e-5


@pytest.mark.parametrize("dims,N", OP_CASES[::2])
def test_apply_A_fp32(dims, N):
    m, o = _pair(dims, N, rho=0.15, seed=N)
    x = inputs.random_vector(m.n_global, seed=200 + N)
    x32 = x.astype(np.float32)
    y_or = o.apply_A(x32.astype(np.float64), 0.1, 0)
    y = m.apply_A(_to_dev(x32, torch.float32), lam=0.1).cpu().numpy().astype(np.float64)
    assert _rel(y, y_or) <= 2e-5


@pytest.mark.parametrize("dims,N", OP_CASES)
@pytest.mark.parametrize("variant", hb.VARIANTS_F64X)
def test_apply_A_double_float(dims, N, variant):
    """HB_F64X: FP64 data, element kernel in double-float arithmetic
    (~47-bit significand): same 1e-12 bar as the FP64 operator, in each
    block shape the double-float kernel is built in."""
    m, o = _pair(dims, N, rho=0.2, seed=N + 5)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64X, variant)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 0)  # the FP64 slot does not steer HB_F64X
    x = inputs.random_vector(m.n_global, seed=500 + N)
    for screen, lam in [(0, 0.1), (1, 0.7)]:
        y_or = o.apply_A(x, lam, screen)
        y = m.apply_A(_to_dev(x), lam=lam, screen=screen, prec=hb.HB_F64X).cpu().numpy()
        assert _rel(y, y_or) <= 1e-12
        assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()


@pytest.mark.parametrize("dims,N,faces", [((3, 2, 2), 3, 0x3F), ((2, 3, 2), 7, 0x15), ((2, 2, 1), 12, 0x2A),
                                           ((4, 3, 3), 5, 0x00), ((1, 2, 2), 15, 0x3F), ((3, 3, 3), 1, 0x07)])
def test_lattice_gather_equals_csr_gather(dims, N, faces):
    """Variant GRID (every local value stored element-major, Z^T by the box's
    lattice arithmetic) sums each DOF's copies in the CSR gather's order and
    association, so y is the same as with the surface-CSR variants, value for
    value, in FP64, FP32 and double-float and both screenings, with partial
    Dirichlet faces; and it meets the oracle's bar."""
    m, o = _pair(dims, N, rho=0.15, seed=N + 40, faces=faces)
    x = inputs.random_vector(m.n_global, seed=700 + N)
    x32 = x.astype(np.float32)
    for screen, lam in [(0, 0.1), (1, 0.6)]:
        for prec, xin in [(hb.HB_F64, _to_dev(x)), (hb.HB_F32, _to_dev(x32, torch.float32)),
                          (hb.HB_F64X, _to_dev(x))]:
            ys = {}
            for v in (3, 67, 131, 139):
                hb.hb_set_kernel_variant(m.handle, prec, v)
                ys[v] = m.apply_A(xin, lam=lam, screen=screen, prec=prec).cpu().numpy()
            for v in (67, 131, 139):
                assert np.array_equal(ys[v], ys[3]), (prec, screen, v, np.abs(ys[v] - ys[3]).max())
        y_or = o.apply_A(x, lam, screen)
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 131)
        y = m.apply_A(_to_dev(x), lam=lam, screen=screen).cpu().numpy()
        assert _rel(y, y_or) <= 1e-12
        assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()


@pytest.mark.parametrize("variant", [131, 139])
def test_cg_with_lattice_gather(variant):
    """CG (Algorithm 1) with p.Ap reduced in the lattice gather: 100 fixed
    iterations follow the oracle's iterates; the mixed solver reaches the FP64
    residual bar."""
    m, o = _pair((4, 4, 4), 7, rho=0.1, seed=0)
    hb.lib().hb_set_cg_fused(m.handle, 1)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F32, variant)
    b = m.rhs(kind=0, seed=0)
    x_or, *_ = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=100)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=100)
    assert res.status == hb.HB_OK and res.iters == 100
    assert _rel(x.cpu().numpy(), x_or) <= 1e-12
    xm, rm = m.cg(b, lam=0.1, rtol=1e-10, max_it=20000, prec=hb.HB_MIXED)
    assert rm.status == hb.HB_OK
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - o.apply_A(xm.cpu().numpy(), 0.1)) <= 1.05e-10 * np.linalg.norm(bn)
    # the double-float operator in the same variant (what its CG uses at N=7)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64X, variant)
    xd, rd = m.cg(b, lam=0.1, rtol=0.0, max_it=100, prec=hb.HB_F64X)
    assert rd.status == hb.HB_OK and rd.iters == 100
    assert _rel(xd.cpu().numpy(), x_or) <= 1e-9


def test_double_float_variant_slot():
    """HB_F64X keeps its own variant: it takes only the shapes its kernel is
    built in, and autotuning it leaves the FP64 choice alone."""
    m, o = _pair((5, 4, 3), 7, rho=0.1, seed=3)
    assert hb.hb_get_kernel_variant(m.handle, hb.HB_F64X) == 3
    for bad in (0, 1, 5, 7, 19, 35):
        with pytest.raises(hb.HBError):
            hb.hb_set_kernel_variant(m.handle, hb.HB_F64X, bad)
    hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 7)
    best, ms = hb.hb_autotune(m.handle, hb.HB_F64X, reps=2)
    assert best in hb.VARIANTS_F64X and sorted(ms) == hb.VARIANTS_F64X
    assert hb.hb_get_kernel_variant(m.handle, hb.HB_F64X) == best
    assert hb.hb_get_kernel_variant(m.handle, hb.HB_F64) == 7
    x = inputs.random_vector(m.n_global, seed=31)
    y = m.apply_A(_to_dev(x), lam=0.1, prec=hb.HB_F64X).cpu().numpy()
    y_or = o.apply_A(x, 0.1, 0)
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()


def test_double_float_split_edge_values():
    """Inputs whose magnitudes leave the float range of the split (tiny,
    huge, zero, negative zero) still give the FP64 operator's result."""
    m, o = _pair((2, 2, 2), 4, rho=0.1, seed=2)
    x = inputs.random_vector(m.n_global, seed=9)
    x[0], x[1], x[2], x[3] = 0.0, -0.0, 1e-300, -3e-41
    x[4], x[5] = 2.0 ** -126, -(2.0 ** -127)
    x *= 1.0
    y_or = o.apply_A(x, 0.1, 0)
    y = m.apply_A(_to_dev(x), lam=0.1, prec=hb.HB_F64X).cpu().numpy()
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()
    big = x * 1e30
    y_or = o.apply_A(big, 0.1, 0)
    y = m.apply_A(_to_dev(big), lam=0.1, prec=hb.HB_F64X).cpu().numpy()
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()


def test_cg_double_float_matches_oracle():
    """CG (Algorithm 1) with the double-float operator: 50 fixed iterations
    agree with the oracle's iterates as closely as the FP64 path does."""
    m, o = _pair((4, 3, 3), 5, rho=0.15, seed=4)
    b = m.rhs(kind=0, seed=4)
    x_or, it_or, rel_or, st_or = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=50)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=50, prec=hb.HB_F64X)
    assert res.status == hb.HB_OK and res.iters == 50
    assert _rel(x.cpu().numpy(), x_or) <= 1e-9
    x2, res2 = m.cg(b, lam=0.1, rtol=1e-10, max_it=5000, prec=hb.HB_F64X)
    assert res2.status == hb.HB_OK and res2.rel_res <= 1e-10
    # the stop is taken on the true residual with the FP64 operator
    r = b - m.apply_A(x2, lam=0.1)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1.01e-10


def test_apply_A_reproducible_and_linear():
    m, o = _pair((4, 4, 3), 5, rho=0.2, seed=3)
    x = _to_dev(inputs.random_vector(m.n_global, seed=1))
    z = _to_dev(inputs.random_vector(m.n_global, seed=2))
    y1 = m.apply_A(x, lam=0.3)
    y2 = m.apply_A(x, lam=0.3)
    assert torch.equal(y1, y2)  # bitwise: fixed summation order, no atomics
    yz = m.apply_A(z, lam=0.3)
    ysum = m.apply_A(x + 2 * z, lam=0.3)
    assert torch.linalg.norm(ysum - (y1 + 2 * yz)) <= 1e-13 * torch.linalg.norm(ysum)
    # symmetry x.Az = z.Ax
    a, b = m.dot(x, yz), m.dot(z, y1)
    assert abs(a - b) <= 1e-12 * abs(a)


def test_apply_A_empty_and_neumann():
    m = hb.Mesh(1, 1, 1, 1)  # every node on a Dirichlet face: no DOFs
    assert m.n_global == 0
    x = torch.zeros(0, dtype=torch.float64, device="cuda")
    m.apply_A(x, torch.zeros(0, dtype=torch.float64, device="cuda"))
    m2, o2 = _pair((2, 2, 2), 3, rho=0.2, faces=0)
    one = torch.ones(m2.n_global, dtype=torch.float64, device="cuda")
    y = m2.apply_A(one, lam=0.0)
    assert y.abs().max().item() < 1e-12  # S 1 = 0 without Dirichlet faces


def test_invalid_arguments():
    for bad in [dict(N=0), dict(N=16), dict(perturb=0.5), dict(ex=0)]:
        kw = dict(ex=2, ey=2, ez=2, N=3, perturb=0.1)
        kw.update(bad)
        with pytest.raises(hb.HBError) as ei:
            hb.Mesh(kw["ex"], kw["ey"], kw["ez"], kw["N"], perturb=kw["perturb"])
        assert ei.value.status == hb.HB_ERR_ARG
    m = hb.Mesh(2, 2, 2, 2)
    x = m.vec()
    with pytest.raises(hb.HBError):
        hb.hb_apply_A(m.handle, hb.HB_F64, 5, 0.0, x.data_ptr(), x.data_ptr() + 8)
    with pytest.raises(hb.HBError):  # x and y overlap
        hb.hb_apply_A(m.handle, hb.HB_F64, 0, 0.0, x.data_ptr(), x.data_ptr())


def test_geometry_error_on_inverted_elements():
    """A perturbation that the oracle finds inverts an element must be refused."""
    found = None
    for seed in range(200):
        o = orc.Mesh(3, 3, 3, 2, rho=0.49, seed=seed)
        if o.min_detJ <= 0:
            found = seed
            break
    if found is None:
        pytest.skip("no inverted element among the seeds tried")
    with pytest.raises(hb.HBError) as ei:
        hb.Mesh(3, 3, 3, 2, perturb=0.49, seed=found)
    assert ei.value.status == hb.HB_ERR_GEOMETRY


# ---------------------------------------------------------------- dot and rhs

@pytest.mark.parametrize("n_dims,N", [((3, 3, 3), 5), ((8, 8, 8), 7), ((2, 2, 2), 1)])
def test_dot(n_dims, N):
    m = hb.Mesh(*n_dims, N)
    a = inputs.random_vector(m.n_global, 5, "normal")
    b = inputs.random_vector(m.n_global, 6, "normal")
    exact = math.fsum((a * b).tolist())
    got = m.dot(_to_dev(a), _to_dev(b))
    assert abs(got - exact) <= 1e-14 * np.abs(a * b).sum()
    a32, b32 = a.astype(np.float32), b.astype(np.float32)
    exact32 = math.fsum((a32.astype(np.float64) * b32.astype(np.float64)).tolist())
    got32 = m.dot(_to_dev(a32, torch.float32), _to_dev(b32, torch.float32))
    assert abs(got32 - exact32) <= 1e-13 * np.abs(a32.astype(np.float64) * b32).sum()


def test_rhs_uniform_bit_exact_and_manufactured():
    m, o = _pair((3, 2, 4), 5, rho=0.2, seed=11)
    b = m.rhs(kind=0, seed=9).cpu().numpy()
    np.testing.assert_array_equal(b, o.rhs(kind=0, seed=9))
    bm = m.rhs(kind=1, lam=0.25).cpu().numpy()
    bo = o.rhs(kind=1, lam=0.25)
    assert np.abs(bm - bo).max() <= 1e-13 * np.abs(bo).max()


# ---------------------------------------------------------------- CG

def test_cg_fixed_100_iterations_small_box():
    """4x4x4 elements, N=7, rho=0.1, lambda=0.1, uniform rhs, 100 iterations."""
    m, o = _pair((4, 4, 4), 7, rho=0.1, seed=0)
    b_or = o.rhs(kind=0, seed=0)
    b = m.rhs(kind=0, seed=0)
    np.testing.assert_array_equal(b.cpu().numpy(), b_or)
    x_or, it_or, rel_or, st_or, hist = o.cg(b_or, 0.1, rtol=0.0, max_it=100, history=True)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=100)
    assert res.status == hb.HB_OK and res.iters == 100 and it_or == 100
    assert _rel(x.cpu().numpy(), x_or) <= 1e-12
    # This box is well conditioned: after 100 iterations the recursive residual
    # r.r is ~1e-26 relative, ten orders below what the true residual can reach
    # in FP64. There each step's rounding perturbs it relatively, so the two
    # recursions agree to ~1e-8 relative, not to 1e-12 (x above does).
    assert abs(res.rel_res - rel_or) <= 1e-7 * rel_or
    r_true = b_or - o.apply_A(x.cpu().numpy(), 0.1)
    assert np.linalg.norm(r_true) <= 1e-13 * np.linalg.norm(b_or)


@pytest.mark.parametrize("N,lam,screen", [(3, 0.1, 0), (7, 0.0, 0), (5, 1.0, 1)])
def test_cg_converged(N, lam, screen):
    m, o = _pair((3, 3, 3), N, rho=0.2, seed=4)
    b = m.rhs(kind=0, seed=2)
    x_or, it_or, rel_or, st_or = o.cg(b.cpu().numpy(), lam, rtol=1e-10, max_it=5000, screen=screen)
    x, res = m.cg(b, lam=lam, rtol=1e-10, max_it=5000, screen=screen)
    assert res.status == hb.HB_OK and st_or == 0
    assert res.rel_res <= 1e-10 and rel_or <= 1e-10
    r = b.cpu().numpy() - o.apply_A(x.cpu().numpy(), lam, screen)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(b.cpu().numpy())
    assert _rel(x.cpu().numpy(), x_or) <= 10 * 1e-10 * max(1.0, it_or / 100)


@pytest.mark.parametrize("N,lam", [(3, 0.1), (7, 0.0), (9, 10.0)])
def test_cg_mixed_precision_reaches_fp64_residual(N, lam):
    m, o = _pair((3, 3, 2), N, rho=0.2, seed=5)
    b = m.rhs(kind=0, seed=3)
    x, res = m.cg(b, lam=lam, rtol=1e-10, max_it=20000, prec=hb.HB_MIXED, inner_rtol=1e-4)
    assert res.status == hb.HB_OK, (res.status, res.rel_res, res.iters, res.outer_iters)
    bn = b.cpu().numpy()
    r = bn - o.apply_A(x.cpu().numpy(), lam)
    assert np.linalg.norm(r) <= 1.01e-10 * np.linalg.norm(bn)
    x_or, *_ = o.cg(bn, lam, rtol=1e-12, max_it=20000)
    err = _rel(x.cpu().numpy(), x_or)
    print(f"mixed N={N} lam={lam}: outer {res.outer_iters} inner {res.iters} err vs oracle {err:.2e}")
    assert err <= 1e-6


@pytest.mark.parametrize("prec,precond", [(hb.HB_F64, 0), (hb.HB_F64, 1), (hb.HB_F64X, 0)])
def test_stepwise_cg_equals_one_call(prec, precond):
    """hb_cg_begin + hb_cg_iterate (in pieces) + hb_cg_finish gives the same
    iterate, bit for bit, as hb_cg_solve with the same iteration count; the
    iteration count never passes max_it."""
    m, o = _pair((3, 3, 2), 5, rho=0.1, seed=8)
    hb.lib().hb_set_cg_fused(m.handle, 1)  # the launched kernels (the stepwise form never fuses)
    b = m.rhs(kind=0, seed=8)
    x1, r1 = m.cg(b, lam=0.1, rtol=0.0, max_it=20, prec=prec, precond=precond)
    x2 = m.vec()
    m.cg_begin(b, x2, lam=0.1, rtol=0.0, max_it=20, prec=prec, precond=precond)
    m.cg_iterate(7)
    m.cg_iterate(5)
    m.cg_iterate(50)
    r2 = m.cg_finish()
    assert r2.iters == 20 and r2.status == hb.HB_OK
    assert torch.equal(x1, x2)
    assert r2.rel_res == r1.rel_res
    with pytest.raises(hb.HBError):
        m.cg_iterate(1)  # finished: no solve begun


@pytest.mark.parametrize("dims,N", [((12, 12, 12), 1), ((3, 2, 2), 3), ((4, 4, 4), 7), ((2, 2, 3), 10), ((2, 1, 2), 15)])
def test_fused_cg_matches_oracle_and_launched_path(dims, N):
    """The one-kernel CG (cooperative launch, grid-wide barriers) follows the
    oracle's iterates and agrees with the launched kernels to rounding."""
    m, o = _pair(dims, N, rho=0.15, seed=N + 20)
    b = m.rhs(kind=0, seed=N)
    x_or, *_ = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=40)
    hb.lib().hb_set_cg_fused(m.handle, 2)
    x_f, r_f = m.cg(b, lam=0.1, rtol=0.0, max_it=40)
    hb.lib().hb_set_cg_fused(m.handle, 1)
    x_l, r_l = m.cg(b, lam=0.1, rtol=0.0, max_it=40)
    assert (r_f.iters, r_f.status) == (r_l.iters, r_l.status) == (40, hb.HB_OK)
    assert _rel(x_f.cpu().numpy(), x_or) <= 1e-11
    assert _rel(x_f.cpu().numpy(), x_l.cpu().numpy()) <= 1e-12
    assert abs(r_f.rel_res - r_l.rel_res) <= 1e-8 * r_l.rel_res
    # converged solve and repeatability
    hb.lib().hb_set_cg_fused(m.handle, 2)
    x1, q1 = m.cg(b, lam=0.1, rtol=1e-10, max_it=5000)
    x2, q2 = m.cg(b, lam=0.1, rtol=1e-10, max_it=5000)
    assert q1.status == hb.HB_OK and q1.rel_res <= 1e-10 and torch.equal(x1, x2)
    bn = b.cpu().numpy()
    assert np.linalg.norm(bn - o.apply_A(x1.cpu().numpy(), 0.1)) <= 1.05e-10 * np.linalg.norm(bn)


def test_fused_cg_breakdown_and_zero_rhs():
    m, _ = _pair((2, 2, 2), 4, rho=0.1, seed=3)
    hb.lib().hb_set_cg_fused(m.handle, 2)
    x, res = m.cg(m.vec(), lam=0.1, rtol=1e-10, max_it=50)
    assert res.iters == 0 and res.status == hb.HB_OK and float(torch.abs(x).max()) == 0.0
    b = m.rhs(kind=0, seed=1)
    x, res = m.cg(b, lam=-1e6, rtol=1e-10, max_it=50)
    assert res.status == hb.HB_ERR_BREAKDOWN
    assert hb.lib().hb_set_cg_fused(m.handle, 3) == hb.HB_ERR_ARG


def test_cg_zero_rhs_and_breakdown():
    m = hb.Mesh(2, 2, 2, 3)
    b = m.vec()
    x, res = m.cg(b, lam=0.1, rtol=1e-10, max_it=50)
    assert res.iters == 0 and res.status == hb.HB_OK and x.abs().max().item() == 0
    b = m.rhs(kind=0, seed=1)
    x, res = m.cg(b, lam=-1e6, rtol=1e-10, max_it=50)
    assert res.status == hb.HB_ERR_BREAKDOWN


def test_cg_non_finite_rhs_is_a_breakdown():
    """A NaN or infinity in b stops every CG form at once with
    HB_ERR_BREAKDOWN instead of returning HB_OK with a NaN residual (a fault
    made on the host: the input)."""
    m = hb.Mesh(3, 3, 2, 5, perturb=0.1, seed=3)
    for bad in (float("nan"), float("inf")):
        b = m.rhs(kind=0, seed=2)
        b[7] = bad
        for fused in (1, 2):
            hb.lib().hb_set_cg_fused(m.handle, fused)
            x, res = m.cg(b, lam=0.1, rtol=1e-10, max_it=50)
            assert res.status == hb.HB_ERR_BREAKDOWN and res.iters == 0, (bad, fused, res.status)
        hb.lib().hb_set_cg_fused(m.handle, 0)
        for kw in ({"precond": 1}, {"prec": hb.HB_MIXED}, {"prec": hb.HB_F64X}):
            x, res = m.cg(b, lam=0.1, rtol=1e-10, max_it=50, **kw)
            assert res.status == hb.HB_ERR_BREAKDOWN, (bad, kw, res.status)
    # the mesh is still usable afterwards
    b = m.rhs(kind=0, seed=2)
    x, res = m.cg(b, lam=0.1, rtol=1e-10, max_it=2000)
    assert res.status == hb.HB_OK and res.rel_res <= 1e-10


def test_autotune_keeps_parity(tmp_path):
    from paper_2202_12477_gb300 import autotune
    m, o = _pair((3, 3, 2), 6, rho=0.2, seed=8)
    chosen = autotune.tune_mesh(m, path=str(tmp_path / "cache.json"), reps=2)
    assert chosen[hb.HB_F64] in hb.VARIANTS and chosen[hb.HB_F32] in hb.VARIANTS
    assert hb.hb_get_kernel_variant(m.handle, hb.HB_F64) == chosen[hb.HB_F64]
    # the cached choice is reused on a new mesh of the same degree
    m2 = hb.Mesh(2, 2, 2, 6, perturb=0.1)
    again = autotune.tune_mesh(m2, path=str(tmp_path / "cache.json"))
    assert again == chosen
    x = inputs.random_vector(m.n_global, seed=5)
    assert _rel(m.apply_A(_to_dev(x), lam=0.1).cpu().numpy(), o.apply_A(x, 0.1)) <= 1e-12


def test_csr_store_variant_survives_rebuilds():
    """The CSR-position store's array is built when the variant is set and
    freed by the autotuner when unused; captured CG runs that used it are
    dropped, so CG after set -> autotune -> set again stays correct."""
    m, o = _pair((3, 3, 3), 5, rho=0.15, seed=12)
    b = m.rhs(kind=0, seed=12)
    x_or, *_ = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=20)
    for variant in (67, 75):
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
        x, r = m.cg(b, lam=0.1, rtol=0.0, max_it=20)
        assert _rel(x.cpu().numpy(), x_or) <= 1e-11
        hb.hb_autotune(m.handle, hb.HB_F64, reps=1)
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, 3)
        hb.hb_autotune(m.handle, hb.HB_F32, reps=1)
        hb.hb_set_kernel_variant(m.handle, hb.HB_F64, variant)
        x2, r2 = m.cg(b, lam=0.1, rtol=0.0, max_it=20)
        assert torch.equal(x, x2)


# ---------------------------------------------------------------- Jacobi preconditioner

@pytest.mark.parametrize("dims,N,rho,lam,screen", [((3, 2, 2), 3, 0.2, 0.1, 0), ((2, 2, 3), 6, 0.25, 0.7, 1),
                                                   ((2, 2, 2), 9, 0.1, 0.0, 0)])
def test_diagonal_matches_oracle(dims, N, rho, lam, screen):
    m, o = _pair(dims, N, rho=rho, seed=N)
    d = m.diag_A(lam=lam, screen=screen)
    d_or = o.diag_A(lam, screen)
    assert np.abs(d - d_or).max() <= 1e-13 * np.abs(d_or).max()


def test_pcg_fixed_iterations_match_oracle():
    m, o = _pair((3, 3, 3), 5, rho=0.25, seed=3)
    b = m.rhs(kind=0, seed=5)
    x_or, it_or, rel_or, st_or = o.cg(b.cpu().numpy(), 0.1, rtol=0.0, max_it=30, precond=1)
    x, res = m.cg(b, lam=0.1, rtol=0.0, max_it=30, precond=1)
    assert res.iters == 30 and it_or == 30 and res.status == hb.HB_OK
    assert _rel(x.cpu().numpy(), x_or) <= 1e-12
    assert abs(res.rel_res - rel_or) <= 1e-9 * rel_or


@pytest.mark.parametrize("prec", [hb.HB_F64, hb.HB_MIXED])
def test_pcg_converges_with_fewer_iterations(prec):
    m, o = _pair((4, 3, 3), 7, rho=0.2, seed=6)
    b = m.rhs(kind=0, seed=6)
    x0, r0 = m.cg(b, lam=0.0, rtol=1e-10, max_it=20000, prec=prec, precond=0)
    x1, r1 = m.cg(b, lam=0.0, rtol=1e-10, max_it=20000, prec=prec, precond=1)
    assert r0.status == hb.HB_OK and r1.status == hb.HB_OK
    assert r1.iters < r0.iters
    bn = b.cpu().numpy()
    r = bn - o.apply_A(x1.cpu().numpy(), 0.0)
    assert np.linalg.norm(r) <= 1.05e-10 * np.linalg.norm(bn)
