"""Python handle on the plain-C FP64 oracle (``hb_oracle.c``).

TEST INFRASTRUCTURE. Only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module. It builds ``hb_oracle.c`` with gcc
(``-O2 -ffp-contract=off``, OpenMP for the independent per-element loop) and
exposes its routines on numpy arrays. It imports nothing from the CUDA library.

What each routine computes, with the passage of hipBone (arXiv 2202.12477) it
follows, is stated in ``hb_oracle.c``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hb_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (skipped if up to date)."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC",
               "-shared", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.c_void_p
        lib.or_u01.restype = C.c_double
        lib.or_u01.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
        lib.or_splitmix64.restype = C.c_uint64
        lib.or_splitmix64.argtypes = [C.c_uint64]
        lib.or_gll.argtypes = [C.c_int, P, P]
        lib.or_deriv.argtypes = [C.c_int, P, P]
        lib.or_mesh_create.restype = P
        lib.or_mesh_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double,
                                       C.c_uint64, C.c_uint]
        lib.or_mesh_free.argtypes = [P]
        lib.or_mesh_sizes.argtypes = [P, P]
        lib.or_mesh_min_detJ.restype = C.c_double
        lib.or_mesh_min_detJ.argtypes = [P]
        for name in ("or_mesh_copy_l2g", "or_mesh_copy_coords", "or_mesh_copy_vertices"):
            getattr(lib, name).argtypes = [P, P]
        lib.or_mesh_copy_geo.argtypes = [P, P, P]
        lib.or_mesh_copy_ref.argtypes = [P, P, P, P]
        lib.or_apply_A.argtypes = [P, C.c_int, C.c_double, P, P]
        lib.or_rhs.argtypes = [P, C.c_int, C.c_uint64, C.c_double, P]
        lib.or_cg.argtypes = [P, C.c_int, C.c_double, P, P, C.c_double, C.c_int,
                              P, P, P]
        lib.or_num_threads.restype = C.c_int
        lib.or_diag_A.argtypes = [P, C.c_int, C.c_double, P]
        lib.or_pcg.argtypes = [P, C.c_int, C.c_double, P, P, C.c_double, C.c_int, C.c_int, P, P, P]
        lib.or_apply_A_rows.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_uint64, C.c_uint,
                                        C.c_int, C.c_double, P, C.c_int64, P, P]
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def u01(seed: int, stream: int, idx: int) -> float:
    return _load().or_u01(seed, stream, idx)


def splitmix64(s: int) -> int:
    return _load().or_splitmix64(s)


def gll(N: int):
    """GLL nodes and weights for degree N (ascending nodes)."""
    xi = np.zeros(N + 1)
    w = np.zeros(N + 1)
    if _load().or_gll(N, _ptr(xi), _ptr(w)) != 0:
        raise ValueError("N must be >= 1")
    return xi, w


def deriv(N: int) -> np.ndarray:
    """D[i, j] = l_j'(xi_i) on the GLL nodes of degree N."""
    xi, _ = gll(N)
    D = np.zeros((N + 1, N + 1))
    _load().or_deriv(N, _ptr(xi), _ptr(D))
    return D


def apply_A_rows(dims, N, rho, seed, x, rows, lam, screen=0, faces=0x3F):
    """(A x)[rows] for the box, built element by element for the requested DOFs
    only (no full mesh): for checks at sizes the full oracle cannot hold."""
    x = np.ascontiguousarray(x, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.zeros(len(rows))
    if _load().or_apply_A_rows(dims[0], dims[1], dims[2], N, rho, seed, faces, screen, lam, _ptr(x),
                               len(rows), _ptr(rows), _ptr(out)) != 0:
        raise ValueError("bad row or allocation failure")
    return out


def num_threads() -> int:
    return _load().or_num_threads()


ALL_FACES = 0x3F


class Mesh:
    """Box of Ex x Ey x Ez hexahedra of degree N, as the oracle builds it."""

    def __init__(self, Ex, Ey, Ez, N, rho=0.0, seed=0, faces=ALL_FACES):
        lib = _load()
        self._h = lib.or_mesh_create(Ex, Ey, Ez, N, rho, seed, faces)
        if not self._h:
            raise MemoryError("oracle mesh creation failed")
        s = np.zeros(3, dtype=np.int64)
        lib.or_mesh_sizes(self._h, _ptr(s))
        self.E, self.n_local, self.n_global = (int(v) for v in s)
        self.Ex, self.Ey, self.Ez, self.N = Ex, Ey, Ez, N
        self.n = N + 1
        self.rho, self.seed, self.faces = rho, seed, faces

    def close(self):
        if self._h:
            _load().or_mesh_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def min_detJ(self) -> float:
        return _load().or_mesh_min_detJ(self._h)

    def l2g(self) -> np.ndarray:
        out = np.zeros(self.n_local, dtype=np.int32)
        _load().or_mesh_copy_l2g(self._h, _ptr(out))
        return out.reshape(self.E, self.n, self.n, self.n)  # [e][k][j][i]

    def geo(self):
        """(G[e,k,j,i,6] in order rr rs rt ss st tt, Jw[e,k,j,i])."""
        G = np.zeros(6 * self.n_local)
        Jw = np.zeros(self.n_local)
        _load().or_mesh_copy_geo(self._h, _ptr(G), _ptr(Jw))
        n = self.n
        return G.reshape(self.E, n, n, n, 6), Jw.reshape(self.E, n, n, n)

    def coords(self) -> np.ndarray:
        X = np.zeros(3 * self.n_local)
        _load().or_mesh_copy_coords(self._h, _ptr(X))
        n = self.n
        return X.reshape(self.E, n, n, n, 3)

    def vertices(self) -> np.ndarray:
        V = np.zeros(3 * (self.Ex + 1) * (self.Ey + 1) * (self.Ez + 1))
        _load().or_mesh_copy_vertices(self._h, _ptr(V))
        return V.reshape(self.Ez + 1, self.Ey + 1, self.Ex + 1, 3)

    def ref(self):
        n = self.n
        xi, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
        _load().or_mesh_copy_ref(self._h, _ptr(xi), _ptr(w), _ptr(D))
        return xi, w, D

    def apply_A(self, x: np.ndarray, lam: float, screen: int = 0) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        assert x.shape == (self.n_global,)
        y = np.zeros(self.n_global)
        if _load().or_apply_A(self._h, screen, lam, _ptr(x), _ptr(y)) != 0:
            raise MemoryError("oracle apply_A failed")
        return y

    def rhs(self, kind: int = 0, seed: int = 0, lam: float = 0.0) -> np.ndarray:
        b = np.zeros(self.n_global)
        _load().or_rhs(self._h, kind, seed, lam, _ptr(b))
        return b

    def diag_A(self, lam: float, screen: int = 0) -> np.ndarray:
        d = np.zeros(self.n_global)
        _load().or_diag_A(self._h, screen, lam, _ptr(d))
        return d

    def cg(self, b, lam, rtol=0.0, max_it=100, screen=0, x0=None, history=False, precond=0):
        """Algorithm 1 (precond=1: with the Jacobi preconditioner diag(A)).
        Returns (x, iters, rel_res, status[, r.r history])."""
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(self.n_global) if x0 is None else np.array(x0, dtype=np.float64)
        it = C.c_int(0)
        rel = C.c_double(0.0)
        hist = np.zeros(max_it + 1)
        st = _load().or_pcg(self._h, screen, lam, _ptr(b), _ptr(x), rtol, max_it, precond,
                            C.byref(it), C.byref(rel), _ptr(hist))
        if st == 1:
            raise MemoryError("oracle cg failed")
        out = (x, it.value, rel.value, st)
        if history:
            out = out + (hist[: it.value + 1],)
        return out
