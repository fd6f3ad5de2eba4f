"""Host logic of the partitioned operator (no GPU): hb_part_plan, the
planner hb_part_create runs before it uploads, against a plain Python plan
written from the rules of Sec. 3.3 as the library documents them.

Rules checked, on node maps from the oracle:
  - element ranks are blocks (ex*px//Ex, ey*py//Ey, ez*pz//Ez);
  - a DOF held by one rank belongs to it; a DOF held by c > 1 ranks goes to
    the floor(u01(seed, 3, g) * c)-th of them in ascending rank order
    ("randomly, but fairly");
  - partition order: owners' blocks in rank order, lexicographic inside;
  - a rank's halo DOFs are those its elements hold and another rank owns; it
    sends each owned DOF once to every other rank holding it;
  - halo elements hold at least one shared DOF; interior elements are split
    into halves.
"""
import numpy as np
import pytest

from oracle import oracle as orc
from paper_2202_12477_gb300 import hb


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_2202_12477_gb300 import build
    build.build()


def _plan_py(l2g, dims, N, NG, grid, seed):
    Ex, Ey, Ez = dims
    px, py, pz = grid
    P = px * py * pz
    n3 = (N + 1) ** 3
    l2g = l2g.reshape(-1, n3)
    E = l2g.shape[0]
    erank = np.empty(E, dtype=np.int64)
    for e in range(E):
        ex, ey, ez = e % Ex, (e // Ex) % Ey, e // (Ex * Ey)
        erank[e] = ex * px // Ex + px * (ey * py // Ey + py * (ez * pz // Ez))
    held = [set() for _ in range(NG)]
    for e in range(E):
        for g in l2g[e]:
            if g >= 0:
                held[g].add(int(erank[e]))
    owner = np.empty(NG, dtype=np.int64)
    for g in range(NG):
        hs = sorted(held[g])
        k = 0
        if len(hs) > 1:
            k = min(int(orc.u01(seed, 3, g) * len(hs)), len(hs) - 1)
        owner[g] = hs[k]
    perm = np.concatenate([np.nonzero(owner == r)[0] for r in range(P)]).astype(np.int32)
    counts = np.zeros((P, 8), dtype=np.int64)
    off = 0
    for r in range(P):
        mine = [e for e in range(E) if erank[e] == r]
        halo_el = [e for e in mine if any(g >= 0 and len(held[g]) > 1 for g in l2g[e])]
        nint = len(mine) - len(halo_el)
        holds = set(int(g) for e in mine for g in l2g[e] if g >= 0)
        n_owned = int((owner == r).sum())
        n_halo = sum(1 for g in holds if owner[g] != r)
        owned_shared = [g for g in range(NG) if owner[g] == r and len(held[g]) > 1]
        n_send = sum(len(held[g]) - 1 for g in owned_shared)
        counts[r] = [n_owned, off, n_halo, n_send, nint // 2, len(halo_el), nint - nint // 2, len(owned_shared)]
        off += n_owned
    n_shared = sum(1 for g in range(NG) if len(held[g]) > 1)
    return perm, n_shared, int(counts[:, 2].sum()), counts


CASES = [((3, 2, 2), 2, 0x3F, (2, 1, 1), 0), ((4, 3, 3), 3, 0x3F, (2, 2, 1), 5), ((3, 3, 3), 4, 0x00, (3, 1, 3), 7),
         ((2, 2, 2), 5, 0x15, (2, 2, 2), 1), ((4, 4, 2), 2, 0x3F, (4, 2, 1), 3), ((2, 3, 2), 3, 0x2A, (1, 1, 1), 0),
         ((5, 2, 2), 1, 0x3F, (5, 2, 2), 9)]


@pytest.mark.parametrize("dims,N,faces,grid,seed", CASES)
def test_plan_matches_python_rules(dims, N, faces, grid, seed):
    o = orc.Mesh(*dims, N, rho=0.1, seed=1, faces=faces)
    l2g = o.l2g().reshape(-1)
    perm, n_shared, exch, counts = hb.hb_part_plan(l2g, dims, N, o.n_global, grid, seed)
    perm_py, n_shared_py, exch_py, counts_py = _plan_py(l2g, dims, N, o.n_global, grid, seed)
    assert np.array_equal(perm, perm_py)
    assert n_shared == n_shared_py and exch == exch_py
    assert np.array_equal(counts, counts_py)
    # every value one rank receives, another sends
    assert counts[:, 3].sum() == exch


def test_plan_owner_choice_depends_on_seed_only_for_shared_dofs():
    dims, N, grid = (4, 4, 4), 3, (2, 2, 2)
    o = orc.Mesh(*dims, N, rho=0.1, seed=1)
    l2g = o.l2g().reshape(-1)
    p0, s0, _, c0 = hb.hb_part_plan(l2g, dims, N, o.n_global, grid, 0)
    p1, s1, _, c1 = hb.hb_part_plan(l2g, dims, N, o.n_global, grid, 1)
    assert s0 == s1 and not np.array_equal(p0, p1)
    # element classification and halo element counts do not depend on the owners
    assert np.array_equal(c0[:, 4:7], c1[:, 4:7])


def test_plan_rejects_bad_input():
    dims, N = (2, 2, 2), 2
    o = orc.Mesh(*dims, N)
    l2g = o.l2g().reshape(-1).copy()
    with pytest.raises(hb.HBError):
        hb.hb_part_plan(l2g, dims, N, o.n_global, (3, 1, 1))  # more ranks than elements along x
    with pytest.raises(hb.HBError):
        hb.hb_part_plan(l2g, dims, N, o.n_global - 1, (2, 1, 1))  # an id past n_global
    bad = l2g.copy()
    g = int(bad[bad >= 0][0])
    bad[bad == g] = -1  # a DOF no element holds
    with pytest.raises(hb.HBError):
        hb.hb_part_plan(bad, dims, N, o.n_global, (2, 1, 1))
