"""Host check (no GPU) of the lattice arithmetic the GRID kernel variant uses
for Z^T: on the box mesh, DOF g is the unmasked lattice point
(I, J, K) = (x0 + g mod NXu, y0 + (g / NXu) mod NYu, z0 + g / (NXu NYu)), and
its copies are node (I - N ex, J - N ey, K - N ez) of the elements holding
it: along each axis the one element whose interior holds the coordinate, or
the two on a shared face (lower first). Taken in (z, y, x) order these are
the copies in ascending element order, the order the CSR gathers sum in.
Checked against the oracle's node map (its own enumeration), for every
Dirichlet-face pattern class."""
import numpy as np
import pytest

from oracle import oracle as orc


def _axis(I, N, E):
    q, r = divmod(I, N)
    if r:
        return [(q, r)]
    if q == 0:
        return [(0, 0)]
    if q == E:
        return [(E - 1, N)]
    return [(q - 1, N), (q, 0)]


def _lattice_copies(g, dims, N, faces):
    Ex, Ey, Ez = dims
    x0, y0, z0 = faces & 1 and 1, faces & 4 and 1, faces & 16 and 1
    NXu = N * Ex + 1 - x0 - (1 if faces & 2 else 0)
    NYu = N * Ey + 1 - y0 - (1 if faces & 8 else 0)
    I, J, K = x0 + g % NXu, y0 + (g // NXu) % NYu, z0 + g // (NXu * NYu)
    n = N + 1
    out = []
    for ez, k in _axis(K, N, Ez):
        for ey, j in _axis(J, N, Ey):
            for ex, i in _axis(I, N, Ex):
                out.append(((ex + Ex * (ey + Ey * ez)), i + n * (j + n * k)))
    return out


@pytest.mark.parametrize("dims,N,faces", [((3, 2, 2), 2, 0x3F), ((2, 3, 2), 3, 0x15), ((2, 2, 3), 4, 0x2A),
                                          ((3, 3, 2), 1, 0x00), ((2, 2, 2), 5, 0x07), ((4, 1, 2), 3, 0x38)])
def test_lattice_copies_match_the_node_map(dims, N, faces):
    o = orc.Mesh(*dims, N, rho=0.1, seed=2, faces=faces)
    n3 = (N + 1) ** 3
    l2g = o.l2g().reshape(-1, n3)
    copies = [[] for _ in range(o.n_global)]
    for e in range(l2g.shape[0]):  # ascending element order
        for q in range(n3):
            if l2g[e, q] >= 0:
                copies[l2g[e, q]].append((e, q))
    for g in range(o.n_global):
        lat = _lattice_copies(g, dims, N, faces)
        assert lat == copies[g], (g, lat, copies[g])
        assert [e for e, _ in lat] == sorted(e for e, _ in lat)
    # every local node of an unmasked lattice point is some DOF's copy exactly once
    assert sum(len(c) for c in copies) == int((l2g >= 0).sum())
