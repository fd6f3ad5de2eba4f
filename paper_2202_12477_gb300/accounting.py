"""FLOP and byte models of the operator and the CG iteration (hipBone, arXiv
2202.12477), used to report throughput and roofline fractions.

n = N + 1, E elements, N_L = E n^3 local nodes, N_G global DOFs.
"""
from __future__ import annotations


def op_local_flops(E: int, N: int) -> int:
    """S_L applied to every element: 12 n^4 (the six 1-D derivative sweeps,
    2 n^2 flops per sweep of one line) + 15 n^3 (the metric factors) per
    element (Sec. 2)."""
    n = N + 1
    return E * (12 * n ** 4 + 15 * n ** 3)


def op_flops(E: int, N: int) -> int:
    """The screened operator with the lambda W term: 12 n^4 + 18 n^3 per element
    (Sec. 3.2, numerator of Eq. op_perf)."""
    n = N + 1
    return E * (12 * n ** 4 + 18 * n ** 3)


def nekbone_flops(E: int, N: int) -> int:
    """NekBone's FLOP count per CG iteration, used for every reported FOM:
    12 E n^4 + 34 E n^3 (Eq. nekbone_flops)."""
    n = N + 1
    return E * (12 * n ** 4 + 34 * n ** 3)


def hipbone_cg_flops(E: int, N: int) -> int:
    """hipBone's own count per CG iteration: 12 E n^4 + 19 E n^3 + 10 E N^3
    (Eq. hipbone_flops)."""
    n = N + 1
    return 12 * E * n ** 4 + 19 * E * n ** 3 + 10 * E * N ** 3


def paper_op_bytes(NG: int, NL: int) -> int:
    """Bytes the paper's operator kernel moves with perfect caching of x:
    8 N_G + 68 N_L (Sec. 3.2)."""
    return 8 * NG + 68 * NL


def paper_cg_bytes(NG: int, NL: int) -> int:
    """Bytes per CG iteration in the paper's two-kernel design: 108 N_G + 80 N_L (Sec. 3.5)."""
    return 108 * NG + 80 * NL


def paper_roofline(N: int, B: float, C: float = float("inf")) -> float:
    """Eq. op_perf: R = min(C, (12 n^4 + 18 n^3) / (8 N^3 + 68 n^3) B)."""
    n = N + 1
    return min(C, (12 * n ** 4 + 18 * n ** 3) / (8 * N ** 3 + 68 * n ** 3) * B)


def ax_local_bytes(NG: int, NL: int, esz: int) -> int:
    """Algorithmic bytes of this library's element kernel (identity screening):
    x read once (esz N_G), node map (4 N_L), six metric factors (6 esz N_L) and
    the element-local result written once (esz N_L)."""
    return esz * NG + (4 + 7 * esz) * NL


def ax_min_bytes(NG: int, NL: int, esz: int) -> int:
    """Least bytes any implementation of A x on assembled vectors must move:
    x read and y written once (2 esz N_G), node map and six metric factors
    (4 + 6 esz) N_L. FP64: 16 N_G + 52 N_L; FP32: 8 N_G + 28 N_L."""
    return 2 * esz * NG + (4 + 6 * esz) * NL


def assemble_bytes(NG: int, nnz: int, esz: int) -> int:
    """The Z^T gather: element-local values and CSR columns (esz + 4 per entry),
    row pointers, x and y (4 + 2 esz per DOF)."""
    return (esz + 4) * nnz + (4 + 2 * esz) * NG


def assembled_cg_min_bytes(NG: int, NL: int) -> int:
    """Least bytes of one CG iteration on assembled vectors with p.Ap and r.r
    fused into the kernels that produce their operands: A p (16 N_G + 52 N_L),
    r -= alpha Ap (read r, Ap; write r: 24 N_G), x += alpha p and
    p = r + beta p (read x, p, r; write x, p: 40 N_G) = 80 N_G + 52 N_L."""
    return 80 * NG + 52 * NL


def scattered_cg_min_bytes(NL: int) -> int:
    """The same iteration on scattered vectors (Sec. 2, Sec. 3.1): A p reads
    p_L and the six factors and writes y_L (64 N_L, no node map); the weighted
    p.Ap, fused, still reads the weights (8 N_L); r -= alpha Ap with the
    weighted r.r reads r, Ap, c and writes r (32 N_L); the x, p update moves
    40 N_L: 144 N_L."""
    return 144 * NL


def box_dofs(N: int, Ex: int, Ey: int, Ez: int) -> int:
    """Global DOFs of a box with Dirichlet nodes on all six faces."""
    return (N * Ex - 1) * (N * Ey - 1) * (N * Ez - 1)
