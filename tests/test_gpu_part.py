"""Partitioned operator (the split, overlapped application of Sec. 3.3 with
virtual ranks on one GPU) against the oracle and against the one-mesh
operator.

Checks:
  - the partition: perm is a permutation; every rank's owned block is
    lexicographically ordered; owners of shared DOFs are among the ranks that
    hold them and are spread fairly; the halo exchange delivers exactly x at
    each rank's halo DOFs;
  - y = A x in partition order equals the oracle's A x (permuted) to 1e-12,
    for several rank grids (uneven blocks, one rank, 64 ranks), degrees,
    screening modes and Dirichlet face sets;
  - CG on the partitioned operator follows the oracle's iterates.
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


def _pair(dims, N, rho=0.15, seed=0, faces=0x3F):
    m = hb.Mesh(*dims, N, perturb=rho, seed=seed, faces=faces, fp32=False)
    o = orc.Mesh(*dims, N, rho=rho, seed=seed, faces=faces)
    return m, o


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _holders(o, grid, dims):
    """Ranks holding each lexicographic DOF (set of ints), from the oracle's l2g."""
    Ex, Ey, Ez = dims
    px, py, pz = grid
    n3 = (o.N + 1) ** 3
    l2g = o.l2g().reshape(-1, n3)
    held = [set() for _ in range(o.n_global)]
    for e in range(l2g.shape[0]):
        ex, ey, ez = e % Ex, (e // Ex) % Ey, e // (Ex * Ey)
        r = ex * px // Ex + px * (ey * py // Ey + py * (ez * pz // Ez))
        for g in l2g[e]:
            if g >= 0:
                held[g].add(r)
    return held


CASES = [((4, 3, 3), 3, (2, 1, 1)), ((4, 4, 3), 5, (2, 2, 1)), ((3, 3, 3), 7, (3, 2, 2)),
         ((5, 4, 3), 2, (2, 2, 2)), ((4, 4, 4), 4, (4, 4, 4)), ((3, 2, 2), 6, (1, 1, 1)),
         ((2, 2, 3), 9, (2, 1, 3))]


@pytest.mark.parametrize("dims,N,grid", CASES)
def test_partition_structure(dims, N, grid):
    m, o = _pair(dims, N, seed=N)
    part = hb.Part(m, *grid, seed=5)
    P = grid[0] * grid[1] * grid[2]
    assert part.n_ranks == P and part.n_global == m.n_global
    perm = part.perm.astype(np.int64)
    assert np.array_equal(np.sort(perm), np.arange(m.n_global))
    held = _holders(o, grid, dims)
    off = 0
    for r in range(P):
        ri = part.rank_info(r)
        assert ri.offset == off
        seg = perm[off:off + ri.n_owned]
        assert np.all(np.diff(seg) > 0)  # lexicographic within the rank
        assert all(r in held[g] for g in seg)
        assert ri.n_elem_interior1 + ri.n_elem_halo + ri.n_elem_interior2 > 0
        off += ri.n_owned
    assert off == m.n_global
    shared = [g for g in range(m.n_global) if len(held[g]) > 1]
    assert part.info.n_shared == len(shared)
    # halo DOFs of a rank: those of its elements owned elsewhere
    assert part.info.exchange_values == sum(part.rank_info(r).n_halo for r in range(P))
    assert part.info.exchange_values == sum(part.rank_info(r).n_send for r in range(P))
    part.close()


def test_owner_choice_is_fair():
    """Shared DOFs go uniformly to their holders: on 8 ranks of a 6^3 box at
    N=4, each holder of the two-rank faces gets about half of them."""
    dims, N, grid = (6, 6, 6), 4, (2, 2, 2)
    m, o = _pair(dims, N, seed=1)
    part = hb.Part(m, *grid, seed=11)
    held = _holders(o, grid, dims)
    owner = np.empty(m.n_global, dtype=np.int64)
    off = 0
    for r in range(8):
        ri = part.rank_info(r)
        owner[part.perm[off:off + ri.n_owned]] = r
        off += ri.n_owned
    two = [g for g in range(m.n_global) if len(held[g]) == 2]
    low = sum(1 for g in two if owner[g] == min(held[g]))
    frac = low / len(two)
    assert len(two) > 1000 and abs(frac - 0.5) < 0.05, frac
    # a different seed gives a different (but still valid) choice
    part2 = hb.Part(m, *grid, seed=12)
    assert not np.array_equal(part.perm, part2.perm)
    part.close()
    part2.close()


@pytest.mark.parametrize("dims,N,grid", CASES[:4])
def test_halo_exchange_delivers_owner_values(dims, N, grid):
    m, o = _pair(dims, N, seed=N)
    part = hb.Part(m, *grid, seed=2)
    x_lex = inputs.random_vector(m.n_global, seed=40 + N)
    x = torch.from_numpy(x_lex[part.perm]).cuda()
    held = _holders(o, grid, dims)
    owner = np.empty(m.n_global, dtype=np.int64)
    off = 0
    for r in range(part.n_ranks):
        ri = part.rank_info(r)
        owner[part.perm[off:off + ri.n_owned]] = r
        off += ri.n_owned
    inv = np.empty(m.n_global, dtype=np.int64)
    inv[part.perm] = np.arange(m.n_global)
    for r in range(part.n_ranks):
        h = part.halo_exchange(x, rank=r)
        want = sorted(inv[g] for g in range(m.n_global) if r in held[g] and owner[g] != r)
        assert h.shape[0] == len(want)
        assert np.array_equal(h, x.cpu().numpy()[want])
    part.close()


@pytest.mark.parametrize("dims,N,grid", CASES)
@pytest.mark.parametrize("screen,lam", [(0, 0.1), (1, 0.7)])
def test_part_apply_matches_oracle(dims, N, grid, screen, lam):
    m, o = _pair(dims, N, seed=N + 2)
    part = hb.Part(m, *grid, seed=3)
    x_lex = inputs.random_vector(m.n_global, seed=60 + N)
    y_or = o.apply_A(x_lex, lam, screen)[part.perm]
    y = part.apply_A(torch.from_numpy(x_lex[part.perm]).cuda(), lam=lam, screen=screen).cpu().numpy()
    assert _rel(y, y_or) <= 1e-12
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()
    # the one-mesh operator on the same input
    y1 = m.apply_A(torch.from_numpy(x_lex).cuda(), lam=lam, screen=screen).cpu().numpy()[part.perm]
    assert np.abs(y - y1).max() <= 1e-13 * np.abs(y1).max()
    part.close()


@pytest.mark.parametrize("faces", [0x00, 0x15])
def test_part_apply_partial_dirichlet(faces):
    dims, N, grid = (4, 3, 3), 4, (2, 2, 1)
    m, o = _pair(dims, N, seed=7, faces=faces)
    part = hb.Part(m, *grid, seed=4)
    x_lex = inputs.random_vector(m.n_global, seed=70)
    y_or = o.apply_A(x_lex, 0.2, 0)[part.perm]
    y = part.apply_A(torch.from_numpy(x_lex[part.perm]).cuda(), lam=0.2).cpu().numpy()
    assert np.abs(y - y_or).max() <= 1e-12 * np.abs(y_or).max()
    part.close()


def test_part_apply_reproducible_and_repeatable():
    m, _ = _pair((4, 4, 4), 5, seed=9)
    part = hb.Part(m, 2, 2, 2, seed=1)
    x = torch.from_numpy(inputs.random_vector(m.n_global, seed=80)).cuda()
    y0 = part.apply_A(x, lam=0.1)
    for _ in range(5):
        assert torch.equal(part.apply_A(x, lam=0.1), y0)
    part.close()


def test_part_cg_follows_oracle():
    dims, N, grid = (4, 3, 3), 5, (2, 2, 1)
    m, o = _pair(dims, N, seed=4)
    part = hb.Part(m, *grid, seed=6)
    b_lex = m.rhs(kind=0, seed=4).cpu().numpy()
    x_or, it_or, rel_or, st_or = o.cg(b_lex, 0.1, rtol=0.0, max_it=50)
    b = torch.from_numpy(b_lex[part.perm]).cuda()
    x, res = part.cg(b, lam=0.1, rtol=0.0, max_it=50)
    assert res.status == hb.HB_OK and res.iters == 50
    assert _rel(x.cpu().numpy(), x_or[part.perm]) <= 1e-9
    x2, res2 = part.cg(b, lam=0.1, rtol=1e-10, max_it=5000)
    assert res2.status == hb.HB_OK and res2.rel_res <= 1e-10
    r = b - part.apply_A(x2, lam=0.1)
    assert float(torch.linalg.norm(r) / torch.linalg.norm(b)) <= 1e-9


def test_part_invalid_arguments():
    m, _ = _pair((2, 2, 2), 3)
    with pytest.raises(hb.HBError):
        hb.Part(m, 3, 1, 1)
    with pytest.raises(hb.HBError):
        hb.Part(m, 0, 1, 1)
    part = hb.Part(m, 2, 1, 1)
    with pytest.raises(hb.HBError):
        part.rank_info(2)
    x = part.vec()
    st = hb.lib().hb_part_apply_A(part.handle, 0, 0.1, hb.C.c_void_p(x.data_ptr()), hb.C.c_void_p(x.data_ptr()),
                                  hb._stream_ptr(None))
    assert st == hb.HB_ERR_ARG
    part.close()
