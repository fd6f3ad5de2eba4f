"""Pins for the FP64 oracle: each test checks it against something other than
itself -- a printed value of the paper, a published test vector, a closed form,
an invariant of the mathematics, an independent library routine, or a dense
brute-force construction -- so that a dropped term, a wrong sign or index, or a
transposed operand anywhere in the oracle fails at least one of them.

CPU only (no GPU needed).
"""
import math
import os

import numpy as np
import numpy.polynomial.legendre as npleg
import pytest

from oracle import oracle as orc

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_rows(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append([int(t) for t in line.split()])
    return rows


# ---------------------------------------------------------------- random numbers

def test_splitmix64_published_vector():
    """SplitMix64 (Steele, Lea & Flood 2014): reference outputs for seed 1234567."""
    want = [r[0] for r in _golden_rows("splitmix64_seed1234567.txt")]
    gamma = 0x9E3779B97F4A7C15
    got = [orc.splitmix64((1234567 + k * gamma) % 2**64) for k in range(len(want))]
    assert got == want


def test_u01_range_and_moments():
    u = np.array([orc.u01(7, 2, i) for i in range(20000)])
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.01
    assert abs(u.var() - 1.0 / 12.0) < 0.005
    # streams and seeds give different sequences
    assert orc.u01(7, 1, 5) != orc.u01(7, 2, 5)
    assert orc.u01(7, 1, 5) != orc.u01(8, 1, 5)


# ---------------------------------------------------------------- GLL and D (Sec. 2)

def test_gll_closed_forms():
    """Textbook GLL nodes/weights for N = 1..4."""
    s5, s37 = 1 / math.sqrt(5), math.sqrt(3 / 7)
    cases = {
        1: ([-1, 1], [1, 1]),
        2: ([-1, 0, 1], [1 / 3, 4 / 3, 1 / 3]),
        3: ([-1, -s5, s5, 1], [1 / 6, 5 / 6, 5 / 6, 1 / 6]),
        4: ([-1, -s37, 0, s37, 1], [1 / 10, 49 / 90, 32 / 45, 49 / 90, 1 / 10]),
    }
    for N, (xs, ws) in cases.items():
        xi, w = orc.gll(N)
        np.testing.assert_allclose(xi, xs, rtol=0, atol=1e-15)
        np.testing.assert_allclose(w, ws, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", range(1, 16))
def test_gll_quadrature_exactness(N):
    """GLL with N+1 points integrates x^p exactly for p <= 2N-1, not for p = 2N."""
    xi, w = orc.gll(N)
    assert abs(w.sum() - 2.0) < 1e-14
    for p in range(0, 2 * N):
        exact = 0.0 if p % 2 else 2.0 / (p + 1)
        assert abs(np.dot(w, xi ** p) - exact) < 1e-13, (N, p)
    p = 2 * N
    assert abs(np.dot(w, xi ** p) - 2.0 / (p + 1)) > 1e-10  # ~4^-N, far above rounding


@pytest.mark.parametrize("N", range(2, 16))
def test_gll_nodes_are_roots_of_legendre_derivative(N):
    """Interior GLL nodes against numpy's roots of P_N' (independent routine)."""
    xi, _ = orc.gll(N)
    dP = npleg.Legendre.basis(N).deriv()
    roots = np.sort(dP.roots().real)
    np.testing.assert_allclose(xi[1:-1], roots, rtol=0, atol=1e-13)
    assert xi[0] == -1.0 and xi[-1] == 1.0


@pytest.mark.parametrize("N", range(1, 16))
def test_deriv_differentiates_polynomials(N):
    """D xi^p = p xi^(p-1) for p <= N; rows sum to 0; D_{N-i,N-j} = -D_ij."""
    xi, _ = orc.gll(N)
    D = orc.deriv(N)
    for p in range(0, N + 1):
        want = p * xi ** (p - 1) if p > 0 else np.zeros_like(xi)
        np.testing.assert_allclose(D @ xi ** p, want, rtol=0, atol=1e-13 * N * N)
    np.testing.assert_allclose(D.sum(axis=1), 0.0, atol=1e-12)
    np.testing.assert_allclose(D[::-1, ::-1], -D, rtol=0, atol=1e-13)


@pytest.mark.parametrize("N", range(1, 11))
def test_deriv_vs_numpy_lagrange(N):
    """D_ij = l_j'(xi_i) with l_j built by numpy's polynomial fit (independent)."""
    xi, _ = orc.gll(N)
    D = orc.deriv(N)
    for j in range(N + 1):
        e = np.zeros(N + 1)
        e[j] = 1.0
        lj = np.polynomial.Polynomial.fit(xi, e, N, domain=[-1, 1], window=[-1, 1])
        np.testing.assert_allclose(D[:, j], lj.deriv()(xi), rtol=0, atol=1e-10)


# ---------------------------------------------------------------- mesh and numbering

@pytest.mark.parametrize("row", [r for r in _golden_rows("dof_counts.txt")
                                 if r[1] * r[2] * r[3] * (r[0] + 1) ** 3 <= 2_000_000])
def test_dof_counts_match_paper(row):
    N, Ex, Ey, Ez, NG = row
    m = orc.Mesh(Ex, Ey, Ez, N)
    assert m.n_global == NG
    assert m.n_local == Ex * Ey * Ez * (N + 1) ** 3


def test_numbering_is_lexicographic_and_shared():
    """Global ids follow the lattice, I fastest; shared nodes get one id."""
    N, Ex, Ey, Ez = 2, 3, 2, 2
    m = orc.Mesh(Ex, Ey, Ez, N, faces=0)
    l2g = m.l2g()
    NX, NY = N * Ex + 1, N * Ey + 1
    for ez in range(Ez):
        for ey in range(Ey):
            for ex in range(Ex):
                e = ex + Ex * (ey + Ey * ez)
                for k in range(N + 1):
                    for j in range(N + 1):
                        for i in range(N + 1):
                            I, J, K = N * ex + i, N * ey + j, N * ez + k
                            assert l2g[e, k, j, i] == I + NX * (J + NY * K)
    # partial Dirichlet: only x=0 face masked
    m2 = orc.Mesh(Ex, Ey, Ez, N, faces=1)
    assert m2.n_global == (NX - 1) * NY * (N * Ez + 1)
    assert (m2.l2g()[:, :, :, 0][np.arange(m2.E) % Ex == 0] == -1).all()


def test_vertices_perturbation():
    Ex, Ey, Ez, rho, seed = 3, 4, 2, 0.2, 11
    m = orc.Mesh(Ex, Ey, Ez, 1, rho=rho, seed=seed)
    V = m.vertices()
    h = np.array([1 / Ex, 1 / Ey, 1 / Ez])
    for c in range(Ez + 1):
        for b in range(Ey + 1):
            for a in range(Ex + 1):
                base = np.array([a / Ex, b / Ey, c / Ez])
                off = V[c, b, a] - base
                inside = 0 < a < Ex and 0 < b < Ey and 0 < c < Ez
                if inside:
                    assert (np.abs(off) <= rho * h + 1e-15).all()
                    assert (np.abs(off) > 0).all()
                else:
                    assert (off == 0).all()


# ---------------------------------------------------------------- geometric factors (Sec. 2)

@pytest.mark.parametrize("N", [1, 3, 6])
def test_undeformed_geometry_closed_form(N):
    """Affine box: G diagonal, G_rr = w_i w_j w_k hy hz / (2 hx) etc., Jw = w w w hx hy hz / 8."""
    Ex, Ey, Ez = 2, 3, 4
    m = orc.Mesh(Ex, Ey, Ez, N, rho=0.0)
    G, Jw = m.geo()
    _, w = orc.gll(N)
    W3 = np.einsum("k,j,i->kji", w, w, w)
    hx, hy, hz = 1 / Ex, 1 / Ey, 1 / Ez
    for e in range(m.E):
        np.testing.assert_allclose(G[e, ..., 0], W3 * hy * hz / (2 * hx), rtol=1e-14)
        np.testing.assert_allclose(G[e, ..., 3], W3 * hx * hz / (2 * hy), rtol=1e-14)
        np.testing.assert_allclose(G[e, ..., 5], W3 * hx * hy / (2 * hz), rtol=1e-14)
        for f in (1, 2, 4):
            assert np.abs(G[e, ..., f]).max() < 1e-15
        np.testing.assert_allclose(Jw[e], W3 * hx * hy * hz / 8, rtol=1e-14)


@pytest.mark.parametrize("N,rho", [(2, 0.25), (5, 0.3), (9, 0.1)])
def test_perturbed_volume_is_one(N, rho):
    """sum Jw = |[0,1]^3| = 1: detJ of a trilinear map is degree <= 2 per variable."""
    m = orc.Mesh(3, 3, 3, N, rho=rho, seed=3)
    _, Jw = m.geo()
    assert abs(Jw.sum() - 1.0) < 1e-13
    assert m.min_detJ > 0


def test_coords_are_continuous_across_elements():
    """Every copy of a shared node has the same physical coordinates."""
    m = orc.Mesh(3, 2, 2, 4, rho=0.2, seed=5, faces=0)
    l2g, X = m.l2g().ravel(), m.coords().reshape(-1, 3)
    ref = np.full((m.n_global, 3), np.nan)
    for q, g in enumerate(l2g):
        if np.isnan(ref[g, 0]):
            ref[g] = X[q]
        else:
            np.testing.assert_allclose(X[q], ref[g], rtol=0, atol=1e-15)


# ---------------------------------------------------------------- the operator (Eq. poisson, Eq. stiffness)

def _dense_from_oracle(m, lam, screen=0):
    I = np.eye(m.n_global)
    return np.stack([m.apply_A(I[:, c], lam, screen) for c in range(m.n_global)], axis=1)


def _dense_bruteforce(m, lam, screen=0):
    """Z^T (sum_e Dbold^T G^e Dbold) Z + lambda I, element matrices built
    explicitly with Kronecker products (independent of the sum factorisation)."""
    n = m.n
    _, _, D = m.ref()
    In = np.eye(n)
    # local node index (k, j, i), i fastest: r acts on i, s on j, t on k
    Dr = np.kron(In, np.kron(In, D))
    Ds = np.kron(In, np.kron(D, In))
    Dt = np.kron(D, np.kron(In, In))
    Dops = [Dr, Ds, Dt]
    G, Jw = m.geo()
    l2g = m.l2g().reshape(m.E, -1)
    A = np.zeros((m.n_global, m.n_global))
    idx = {(0, 0): 0, (0, 1): 1, (0, 2): 2, (1, 1): 3, (1, 2): 4, (2, 2): 5}
    for e in range(m.E):
        g = G[e].reshape(-1, 6)
        K = np.zeros((n ** 3, n ** 3))
        for a in range(3):
            for b in range(3):
                f = idx[(min(a, b), max(a, b))]
                K += Dops[a].T @ (g[:, f][:, None] * Dops[b])
        if screen == 1:
            K += lam * np.diag(Jw[e].ravel())
        Z = np.zeros((n ** 3, m.n_global))
        for q, gid in enumerate(l2g[e]):
            if gid >= 0:
                Z[q, gid] = 1.0
        A += Z.T @ K @ Z
    if screen == 0:
        A += lam * np.eye(m.n_global)
    return A


@pytest.mark.parametrize("dims,N,rho,lam,screen", [
    ((1, 1, 1), 1, 0.0, 0.0, 0), ((2, 2, 2), 1, 0.2, 0.1, 0), ((2, 1, 1), 3, 0.0, 0.5, 0),
    ((2, 2, 2), 2, 0.25, 0.1, 0), ((2, 2, 1), 4, 0.2, 1.0, 1), ((2, 2, 2), 3, 0.3, 0.0, 0),
    ((1, 2, 2), 5, 0.1, 10.0, 0), ((2, 2, 2), 6, 0.1, 0.1, 1), ((2, 2, 2), 4, 0.1, 0.1, 0),
])
def test_matrix_free_equals_dense_bruteforce(dims, N, rho, lam, screen):
    """The matrix-free oracle against the explicitly assembled matrix (1-8 elements)."""
    m = orc.Mesh(*dims, N, rho=rho, seed=1, faces=0x3F if N > 1 or dims != (1, 1, 1) else 0)
    if m.n_global == 0:
        pytest.skip("no interior DOFs")
    A0 = _dense_from_oracle(m, lam, screen)
    A1 = _dense_bruteforce(m, lam, screen)
    scale = np.abs(A1).max()
    assert np.abs(A0 - A1).max() <= 1e-13 * scale


def _fem1d(E, N, h):
    """Assembled 1-D stiffness (2/h) D^T W D and lumped mass (h/2) W, Dirichlet rows removed."""
    xi, w = orc.gll(N)
    D = orc.deriv(N)
    Ke = (2.0 / h) * D.T @ np.diag(w) @ D
    Me = (h / 2.0) * np.diag(w)
    nn = N * E + 1
    K = np.zeros((nn, nn))
    M = np.zeros((nn, nn))
    for e in range(E):
        s = slice(N * e, N * e + N + 1)
        K[s, s] += Ke
        M[s, s] += Me
    return K[1:-1, 1:-1], M[1:-1, 1:-1]


@pytest.mark.parametrize("dims,N,lam", [((2, 3, 2), 3, 0.1), ((3, 2, 2), 1, 0.0), ((1, 2, 3), 4, 2.0)])
def test_undeformed_operator_is_kronecker_sum(dims, N, lam):
    """Affine box: S = Mz (x) My (x) Kx + Mz (x) Ky (x) Mx + Kz (x) My (x) Mx."""
    Ex, Ey, Ez = dims
    m = orc.Mesh(Ex, Ey, Ez, N, rho=0.0)
    Kx, Mx = _fem1d(Ex, N, 1 / Ex)
    Ky, My = _fem1d(Ey, N, 1 / Ey)
    Kz, Mz = _fem1d(Ez, N, 1 / Ez)
    S = np.kron(Mz, np.kron(My, Kx)) + np.kron(Mz, np.kron(Ky, Mx)) + np.kron(Kz, np.kron(My, Mx))
    A = S + lam * np.eye(S.shape[0])
    A0 = _dense_from_oracle(m, lam)
    assert np.abs(A0 - A).max() <= 1e-13 * np.abs(A).max()


@pytest.mark.parametrize("N,rho,lam,screen", [(3, 0.2, 0.0, 0), (5, 0.3, 0.1, 0), (4, 0.25, 1.0, 1)])
def test_symmetric_positive_definite(N, rho, lam, screen):
    m = orc.Mesh(2, 2, 2, N, rho=rho, seed=9)
    rng = np.random.default_rng(0)
    x, y = rng.standard_normal(m.n_global), rng.standard_normal(m.n_global)
    xAy, yAx = x @ m.apply_A(y, lam, screen), y @ m.apply_A(x, lam, screen)
    assert abs(xAy - yAx) <= 1e-13 * max(abs(xAy), 1.0) * 10
    A = _dense_from_oracle(m, lam, screen)
    np.linalg.cholesky(0.5 * (A + A.T))  # raises if not SPD


@pytest.mark.parametrize("N,rho", [(2, 0.2), (4, 0.3), (7, 0.1)])
def test_linear_functions_are_integrated_exactly(N, rho):
    """No Dirichlet faces, lambda = 0: S 1 = 0 and (a.x)^T S (b.x) = a.b |Omega| = a.b."""
    m = orc.Mesh(2, 3, 2, N, rho=rho, seed=4, faces=0)
    l2g, X = m.l2g().ravel(), m.coords().reshape(-1, 3)
    Xg = np.zeros((m.n_global, 3))
    Xg[l2g] = X
    one = np.ones(m.n_global)
    assert np.abs(m.apply_A(one, 0.0)).max() < 1e-12
    rng = np.random.default_rng(2)
    a, b = rng.standard_normal(3), rng.standard_normal(3)
    ua, ub = Xg @ a, Xg @ b
    assert abs(ua @ m.apply_A(ub, 0.0) - a @ b) < 1e-12


# ---------------------------------------------------------------- right-hand sides

def test_uniform_rhs_follows_lattice_generator():
    m = orc.Mesh(2, 3, 2, 3, rho=0.1, seed=0)
    b = m.rhs(kind=0, seed=42)
    l2g = m.l2g()
    N, NX, NY = m.N, 3 * 2 + 1, 3 * 3 + 1
    for ez in range(2):
        for ey in range(3):
            for ex in range(2):
                e = ex + 2 * (ey + 3 * ez)
                for (k, j, i) in [(1, 1, 1), (0, 2, 3), (3, 3, 2)]:
                    g = l2g[e, k, j, i]
                    if g < 0:
                        continue
                    lat = (N * ex + i) + NX * ((N * ey + j) + NY * (N * ez + k))
                    assert b[g] == 2.0 * orc.u01(42, 2, lat) - 1.0
    assert b.min() >= -1 and b.max() <= 1 and abs(b.mean()) < 0.1


# ---------------------------------------------------------------- CG (Algorithm 1)

@pytest.mark.parametrize("dims,N,rho,lam", [((2, 2, 2), 3, 0.2, 0.1), ((1, 2, 2), 5, 0.1, 0.0),
                                            ((2, 2, 2), 4, 0.3, 1.0)])
def test_cg_matches_dense_solve(dims, N, rho, lam):
    m = orc.Mesh(*dims, N, rho=rho, seed=2)
    b = m.rhs(kind=0, seed=1)
    A = _dense_bruteforce(m, lam)
    xs = np.linalg.solve(A, b)
    x, it, rel, st = m.cg(b, lam, rtol=1e-12, max_it=5000)
    assert st == 0 and rel <= 1e-12
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)


def test_cg_recursive_residual_tracks_true_residual():
    m = orc.Mesh(2, 2, 2, 4, rho=0.2, seed=2)
    b = m.rhs(kind=0, seed=3)
    for k in (1, 5, 20):
        x, it, rel, st, hist = m.cg(b, 0.1, rtol=0.0, max_it=k, history=True)
        assert it == k and st == 0 and len(hist) == k + 1
        r = b - m.apply_A(x, 0.1)
        assert abs(np.sqrt(r @ r) - np.sqrt(hist[-1])) <= 1e-10 * np.sqrt(b @ b)
    # monotone energy-norm decrease is not guaranteed for r.r, but it must drop overall
    assert hist[-1] < 1e-2 * hist[0]


def test_cg_zero_rhs_and_fixed_iterations():
    m = orc.Mesh(2, 2, 2, 2)
    x, it, rel, st = m.cg(np.zeros(m.n_global), 0.1, rtol=1e-10, max_it=50)
    assert it == 0 and st == 0 and not x.any()
    b = m.rhs(kind=0, seed=0)
    x, it, rel, st = m.cg(b, 0.1, rtol=0.0, max_it=7)
    assert it == 7


def test_cg_breakdown_on_indefinite_operator():
    """lambda far below -lambda_min(S) makes A negative definite: p.Ap < 0 at once."""
    m = orc.Mesh(2, 2, 2, 2)
    b = m.rhs(kind=0, seed=0)
    x, it, rel, st = m.cg(b, -1e6, rtol=1e-10, max_it=50)
    assert st == 2 and it == 0


# ---------------------------------------------------------------- manufactured solution

@pytest.mark.slow
def test_manufactured_solution_converges_spectrally():
    """lambda = 0, u = sin(pi x) sin(pi y) sin(pi z) on 2^3 perturbed elements:
    the nodal error falls exponentially with N."""
    errs = []
    Ns = list(range(2, 13))
    for N in Ns:
        m = orc.Mesh(2, 2, 2, N, rho=0.1, seed=0)
        b = m.rhs(kind=1, lam=0.0)
        x, it, rel, st = m.cg(b, 0.0, rtol=1e-14, max_it=20000)
        l2g, X = m.l2g().ravel(), m.coords().reshape(-1, 3)
        mask = l2g >= 0
        u = np.sin(np.pi * X[mask, 0]) * np.sin(np.pi * X[mask, 1]) * np.sin(np.pi * X[mask, 2])
        errs.append(np.abs(x[l2g[mask]] - u).max())
    errs = np.array(errs)
    slope = np.polyfit(Ns, np.log(errs), 1)[0]
    assert slope < -1.5, errs
    assert errs[-1] < 1e-8, errs
    # every two degrees the error falls
    assert all(errs[i + 2] < errs[i] for i in range(len(errs) - 2)), errs


def test_manufactured_solution_algebraic_rate():
    """Fixed N = 2, refining the (unperturbed) mesh: nodal error ~ h^(N+1) or better."""
    errs = []
    for E in (2, 4, 8):
        m = orc.Mesh(E, E, E, 2)
        b = m.rhs(kind=1, lam=0.0)
        x, it, rel, st = m.cg(b, 0.0, rtol=1e-13, max_it=5000)
        l2g, X = m.l2g().ravel(), m.coords().reshape(-1, 3)
        mask = l2g >= 0
        u = np.prod(np.sin(np.pi * X[mask]), axis=1)
        errs.append(np.abs(x[l2g[mask]] - u).max())
    rates = np.log2(np.array(errs[:-1]) / np.array(errs[1:]))
    assert (rates > 2.5).all(), (errs, rates)


@pytest.mark.parametrize("dims,N,rho,lam,screen,faces", [((3, 2, 2), 3, 0.2, 0.1, 0, 0x3F),
                                                         ((2, 3, 2), 5, 0.25, 0.7, 1, 0x3F),
                                                         ((2, 2, 2), 2, 0.1, 0.0, 0, 0x15),
                                                         ((3, 1, 2), 7, 0.1, 0.3, 1, 0x00)])
def test_sampled_rows_equal_full_operator(dims, N, rho, lam, screen, faces):
    """The row-by-row evaluation (used at sizes the full oracle cannot hold)
    gives exactly the full oracle's rows: same elements, same summation order."""
    m = orc.Mesh(*dims, N, rho=rho, seed=6, faces=faces)
    x = np.random.default_rng(3).standard_normal(m.n_global)
    y = m.apply_A(x, lam, screen)
    rows = np.arange(m.n_global)
    yr = orc.apply_A_rows(dims, N, rho, 6, x, rows, lam, screen, faces)
    np.testing.assert_array_equal(yr, y)


@pytest.mark.parametrize("dims,N,rho,lam,screen", [((2, 2, 2), 3, 0.2, 0.1, 0), ((2, 1, 2), 5, 0.3, 0.7, 1),
                                                   ((1, 2, 2), 2, 0.0, 0.0, 0)])
def test_diagonal_equals_dense_diagonal(dims, N, rho, lam, screen):
    m = orc.Mesh(*dims, N, rho=rho, seed=5)
    A = _dense_bruteforce(m, lam, screen)
    np.testing.assert_allclose(m.diag_A(lam, screen), np.diag(A), rtol=1e-13, atol=0)


@pytest.mark.parametrize("N,lam", [(3, 0.1), (5, 0.0)])
def test_jacobi_pcg_matches_dense_solve(N, lam):
    m = orc.Mesh(2, 2, 2, N, rho=0.25, seed=2)
    b = m.rhs(kind=0, seed=4)
    xs = np.linalg.solve(_dense_bruteforce(m, lam), b)
    x, it, rel, st = m.cg(b, lam, rtol=1e-12, max_it=5000, precond=1)
    assert st == 0 and rel <= 1e-12
    assert np.linalg.norm(x - xs) <= 1e-10 * np.linalg.norm(xs)
    x0, it0, *_ = m.cg(b, lam, rtol=1e-12, max_it=5000, precond=0)
    assert it <= it0  # diagonal scaling never hurts on these meshes
