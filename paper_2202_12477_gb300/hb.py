"""ctypes binding of the C ABI in ``include/hipbone_gb300.h``.

Argument marshalling only: every step of the operator and the solvers runs in
the CUDA library ``_lib/libhbgb300.so``. The functions keep the C names; the
``Mesh`` class is a small convenience owner of a mesh handle that takes torch
CUDA tensors (torch provides device memory and streams, nothing else).

If the library is missing this module raises at import of ``lib()``: there is
no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_lib", "libhbgb300.so")

# hb_status
HB_OK, HB_ERR_ARG, HB_ERR_NOMEM, HB_ERR_CUDA, HB_ERR_GEOMETRY = 0, 1, 2, 3, 4
HB_ERR_BREAKDOWN, HB_ERR_NOT_CONVERGED, HB_ERR_TIMEOUT, HB_ERR_BUSY, HB_ERR_NOT_FOUND = 5, 6, 7, 8, 9
STATUS_NAMES = {0: "HB_OK", 1: "HB_ERR_ARG", 2: "HB_ERR_NOMEM", 3: "HB_ERR_CUDA", 4: "HB_ERR_GEOMETRY",
                5: "HB_ERR_BREAKDOWN", 6: "HB_ERR_NOT_CONVERGED", 7: "HB_ERR_TIMEOUT", 8: "HB_ERR_BUSY",
                9: "HB_ERR_NOT_FOUND"}
# hb_precision
HB_F64, HB_F32, HB_MIXED, HB_F64X = 0, 1, 2, 3
# hb_screen
HB_SCREEN_IDENTITY, HB_SCREEN_MASS = 0, 1
ALL_FACES = 0x3F


class hb_mesh_desc(C.Structure):
    _fields_ = [("ex", C.c_int), ("ey", C.c_int), ("ez", C.c_int), ("N", C.c_int),
                ("perturb", C.c_double), ("seed", C.c_uint64), ("dirichlet_faces", C.c_uint),
                ("keep_fp32_copy", C.c_int)]


class hb_mesh_info_t(C.Structure):
    _fields_ = [("n_local", C.c_int64), ("n_global", C.c_int64), ("n_elem", C.c_int64),
                ("nnz", C.c_int64), ("N", C.c_int), ("l2g", C.c_void_p), ("geo", C.c_void_p),
                ("geo32", C.c_void_p), ("csr_rowptr", C.c_void_p), ("csr_cols", C.c_void_p),
                ("min_detJ", C.c_double), ("device_bytes", C.c_size_t)]


class hb_cg_opts(C.Structure):
    _fields_ = [("prec", C.c_int), ("screen", C.c_int), ("lambda_", C.c_double), ("rtol", C.c_double),
                ("max_it", C.c_int), ("inner_rtol", C.c_double), ("max_outer", C.c_int), ("precond", C.c_int)]


class hb_cg_result(C.Structure):
    _fields_ = [("iters", C.c_int), ("outer_iters", C.c_int), ("rel_res", C.c_double),
                ("time_ms", C.c_double), ("status", C.c_int)]


class hb_server_opts(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("iters_per_launch", C.c_int)]


class hb_server_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("rounds", C.c_int64), ("active", C.c_int), ("pending", C.c_int),
                ("mem_used", C.c_size_t), ("admit_s", C.c_double), ("round_s", C.c_double),
                ("retire_s", C.c_double), ("queue_s", C.c_double), ("build_s", C.c_double),
                ("run_s", C.c_double)]


class hb_part_info_t(C.Structure):
    _fields_ = [("n_ranks", C.c_int), ("n_global", C.c_int64), ("n_shared", C.c_int64),
                ("exchange_values", C.c_int64)]


class hb_part_rank_info_t(C.Structure):
    _fields_ = [("n_owned", C.c_int64), ("offset", C.c_int64), ("n_halo", C.c_int64), ("n_send", C.c_int64),
                ("n_elem_interior1", C.c_int64), ("n_elem_halo", C.c_int64), ("n_elem_interior2", C.c_int64)]


class HBError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


_lib = None

# (name, restype, argtypes) of every exported entry point
_SIGS = [
    ("hb_mesh_create", C.c_int, [C.POINTER(hb_mesh_desc), C.c_void_p, C.POINTER(C.c_void_p)]),
    ("hb_mesh_destroy", C.c_int, [C.c_void_p]),
    ("hb_mesh_info", C.c_int, [C.c_void_p, C.POINTER(hb_mesh_info_t)]),
    ("hb_mesh_copy_l2g", C.c_int, [C.c_void_p, C.c_void_p]),
    ("hb_mesh_copy_geo", C.c_int, [C.c_void_p, C.c_void_p]),
    ("hb_apply_A", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("hb_dot", C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double),
                         C.c_void_p]),
    ("hb_dot_noalloc", C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p,
                                 C.POINTER(C.c_double), C.c_void_p]),
    ("hb_fill_rhs", C.c_int, [C.c_void_p, C.c_int, C.c_uint64, C.c_double, C.c_void_p, C.c_void_p]),
    ("hb_diag_A", C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p]),
    ("hb_cg_solve", C.c_int, [C.c_void_p, C.POINTER(hb_cg_opts), C.c_void_p, C.c_void_p,
                              C.POINTER(hb_cg_result), C.c_void_p]),
    ("hb_u01", C.c_double, [C.c_uint64, C.c_uint64, C.c_uint64]),
    ("hb_set_cg_fused", C.c_int, [C.c_void_p, C.c_int]),
    ("hb_cg_begin", C.c_int, [C.c_void_p, C.POINTER(hb_cg_opts), C.c_void_p, C.c_void_p, C.c_void_p]),
    ("hb_cg_iterate", C.c_int, [C.c_void_p, C.c_int, C.c_void_p]),
    ("hb_cg_finish", C.c_int, [C.c_void_p, C.POINTER(hb_cg_result), C.c_void_p]),
    ("hb_scat_create", C.c_int, [C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    ("hb_scat_destroy", C.c_int, [C.c_void_p]),
    ("hb_scat_scatter", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("hb_scat_apply_A", C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("hb_scat_dot", C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double), C.c_void_p]),
    ("hb_scat_cg_solve", C.c_int, [C.c_void_p, C.POINTER(hb_cg_opts), C.c_void_p, C.c_void_p,
                                   C.POINTER(hb_cg_result), C.c_void_p]),
    ("hb_part_create", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_uint64, C.c_void_p,
                                 C.POINTER(C.c_void_p)]),
    ("hb_part_destroy", C.c_int, [C.c_void_p]),
    ("hb_part_plan", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int64, C.c_int, C.c_int,
                               C.c_int, C.c_uint64, C.c_void_p, C.c_void_p]),
    ("hb_part_info", C.c_int, [C.c_void_p, C.POINTER(hb_part_info_t)]),
    ("hb_part_rank_info", C.c_int, [C.c_void_p, C.c_int, C.POINTER(hb_part_rank_info_t)]),
    ("hb_part_copy_perm", C.c_int, [C.c_void_p, C.c_void_p]),
    ("hb_part_apply_A", C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("hb_part_halo_exchange", C.c_int, [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p]),
    ("hb_part_cg_solve", C.c_int, [C.c_void_p, C.POINTER(hb_cg_opts), C.c_void_p, C.c_void_p,
                                   C.POINTER(hb_cg_result), C.c_void_p]),
    ("hb_server_create", C.c_int, [C.POINTER(hb_server_opts), C.POINTER(C.c_void_p)]),
    ("hb_server_submit", C.c_int, [C.c_void_p, C.POINTER(hb_mesh_desc), C.POINTER(hb_cg_opts), C.c_uint64,
                                   C.c_int, C.POINTER(C.c_int64)]),
    ("hb_server_poll", C.c_int, [C.c_void_p, C.c_int64, C.POINTER(hb_cg_result), C.POINTER(C.c_int64),
                                 C.c_void_p]),
    ("hb_server_stats", C.c_int, [C.c_void_p, C.POINTER(hb_server_stats_t)]),
    ("hb_server_destroy", C.c_int, [C.c_void_p]),
    ("hb_server_inject_round_error", C.c_int, [C.c_void_p]),
    ("hb_tc_selftest", C.c_int, [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    ("hb_set_kernel_variant", C.c_int, [C.c_void_p, C.c_int, C.c_int]),
    ("hb_get_kernel_variant", C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_int)]),
    ("hb_autotune", C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_double, C.c_int, C.POINTER(C.c_int),
                              C.POINTER(C.c_double), C.c_void_p]),
    ("hb_probe", C.c_int, [C.c_int, C.c_int, C.c_size_t, C.c_int, C.POINTER(C.c_double)]),
    ("hb_selftest_wait", C.c_int, [C.c_int, C.POINTER(C.c_int), C.c_void_p]),
    ("hb_kernel_launches", C.c_ulonglong, []),
    ("hb_profile_enable", C.c_int, [C.c_int]),
    ("hb_profile_reset", C.c_int, []),
    ("hb_profile_read", C.c_int, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(C.c_longlong)]),
    ("hb_last_error", C.c_char_p, []),
]


def lib():
    """Load the CUDA library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"CUDA library not built: {LIB_PATH} is missing "
                               "(run paper_2202_12477_gb300.build.build())")
        L = C.CDLL(LIB_PATH)
        for name, res, args in _SIGS:
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def exported_names():
    return [name for name, _, _ in _SIGS]


def _check(status):
    if status != HB_OK:
        raise HBError(status, lib().hb_last_error().decode(errors="replace"))
    return status


def _stream_ptr(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


# ---------------------------------------------------------------- C names

def hb_mesh_create(desc: hb_mesh_desc, stream=None) -> C.c_void_p:
    h = C.c_void_p()
    _check(lib().hb_mesh_create(C.byref(desc), _stream_ptr(stream), C.byref(h)))
    return h


def hb_mesh_destroy(h) -> None:
    _check(lib().hb_mesh_destroy(h))


def hb_mesh_info(h) -> hb_mesh_info_t:
    info = hb_mesh_info_t()
    _check(lib().hb_mesh_info(h, C.byref(info)))
    return info


def hb_apply_A(h, prec, screen, lam, x_ptr, y_ptr, stream=None) -> None:
    _check(lib().hb_apply_A(h, prec, screen, lam, C.c_void_p(x_ptr), C.c_void_p(y_ptr), _stream_ptr(stream)))


def hb_dot(h, prec, a_ptr, b_ptr, out_dev_ptr=None, want_host=True, stream=None):
    out = C.c_double(0.0)
    _check(lib().hb_dot(h, prec, C.c_void_p(a_ptr), C.c_void_p(b_ptr), C.c_void_p(out_dev_ptr or 0),
                        C.byref(out) if want_host else None, _stream_ptr(stream)))
    return out.value if want_host else None


def hb_fill_rhs(h, kind, seed, lam, b_ptr, stream=None) -> None:
    _check(lib().hb_fill_rhs(h, kind, seed, lam, C.c_void_p(b_ptr), _stream_ptr(stream)))


def hb_cg_solve(h, opts: hb_cg_opts, b_ptr, x_ptr, stream=None, check=True) -> hb_cg_result:
    res = hb_cg_result()
    st = lib().hb_cg_solve(h, C.byref(opts), C.c_void_p(b_ptr), C.c_void_p(x_ptr), C.byref(res),
                           _stream_ptr(stream))
    if check and st not in (HB_OK, HB_ERR_NOT_CONVERGED, HB_ERR_BREAKDOWN):
        _check(st)
    return res


def hb_u01(seed, stream, idx) -> float:
    return lib().hb_u01(seed, stream, idx)


HB_VARIANT_PENCIL, HB_VARIANT_EVEN_ODD, HB_VARIANT_EB2, HB_VARIANT_ONE, HB_VARIANT_TMA, HB_VARIANT_WS = \
    1, 2, 4, 8, 16, 32
HB_VARIANT_CSR = 64
HB_VARIANT_GRID = 128
HB_VARIANT_TC = 256  # tensor-core element kernel (HB_F64, N = 7)
VARIANTS_TC = [HB_VARIANT_TC, HB_VARIANT_TC | HB_VARIANT_CSR]  # alone, and with the CSR-position store
VARIANTS = [0, 1, 3, 5, 7, 11, 19, 35, 67, 75, 131, 139]  # every valid combination of the pencil flags
VARIANTS_F64X = [3, 11, 67, 75, 131, 139]  # the shapes the double-float kernel is built in


def hb_set_kernel_variant(h, prec, variant) -> None:
    _check(lib().hb_set_kernel_variant(h, prec, variant))


def hb_get_kernel_variant(h, prec) -> int:
    v = C.c_int(-1)
    _check(lib().hb_get_kernel_variant(h, prec, C.byref(v)))
    return v.value


def hb_autotune(h, prec, screen=HB_SCREEN_IDENTITY, lam=0.1, reps=5, stream=None):
    """Times every kernel variant on this mesh, keeps the fastest; returns
    (best variant, {variant: ms})."""
    best = C.c_int(-1)
    ms = (C.c_double * 512)(*([-1.0] * 512))
    _check(lib().hb_autotune(h, prec, screen, lam, reps, C.byref(best), ms, _stream_ptr(stream)))
    return best.value, {v: ms[v] for v in VARIANTS + VARIANTS_TC if ms[v] >= 0}


HB_PROBE_STREAM81_FP, HB_PROBE_STREAM81_BITS, HB_PROBE_COPY, HB_PROBE_FMA = 0, 1, 2, 3
HB_PROBE_DMMA, HB_PROBE_DMMA_FMA, HB_PROBE_CVT64 = 4, 5, 6


def hb_probe(kind, prec=HB_F64, nbytes=4 << 30, reps=5) -> float:
    """Best rate of a calibration probe: GB/s (stream, copy) or GFLOP/s (FMA)."""
    r = C.c_double(0.0)
    _check(lib().hb_probe(kind, prec, nbytes, reps, C.byref(r)))
    return r.value


def hb_selftest_wait(which, stream=None) -> int:
    """Runs a kernel whose bounded wait (0: mbarrier, 1: grid barrier) can
    never complete; returns the status it reported (HB_ERR_TIMEOUT expected)."""
    st = C.c_int(-1)
    _check(lib().hb_selftest_wait(which, C.byref(st), _stream_ptr(stream)))
    return st.value


def hb_kernel_launches() -> int:
    return lib().hb_kernel_launches()


def hb_profile_enable(on: bool) -> None:
    _check(lib().hb_profile_enable(1 if on else 0))


def hb_profile_reset() -> None:
    _check(lib().hb_profile_reset())


def hb_profile_read(name: str):
    """(total device ms, launches) recorded for kernel `name`."""
    ms = C.c_double(0.0)
    cnt = C.c_longlong(0)
    _check(lib().hb_profile_read(name.encode(), C.byref(ms), C.byref(cnt)))
    return ms.value, cnt.value


# ---------------------------------------------------------------- convenience owner

class Mesh:
    """Owns one hb_mesh; vectors are torch CUDA tensors of length n_global."""

    def __init__(self, ex, ey, ez, N, perturb=0.0, seed=0, faces=ALL_FACES, fp32=True, stream=None):
        self.desc = hb_mesh_desc(ex, ey, ez, N, perturb, seed, faces, 1 if fp32 else 0)
        self.handle = hb_mesh_create(self.desc, stream)
        self.info = hb_mesh_info(self.handle)
        self.n_global = self.info.n_global
        self.n_local = self.info.n_local
        self.E = self.info.n_elem
        self.N = N

    def close(self):
        if getattr(self, "handle", None):
            hb_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self, dtype=None):
        import torch
        return torch.zeros(self.n_global, dtype=dtype or torch.float64, device="cuda")

    def apply_A(self, x, y=None, lam=0.0, screen=HB_SCREEN_IDENTITY, stream=None, prec=None):
        """y = A x. The precision follows x's dtype (float64: HB_F64, float32:
        HB_F32) unless `prec` is given (HB_F64X takes float64 vectors)."""
        import torch
        if prec is None:
            prec = HB_F64 if x.dtype == torch.float64 else HB_F32
        assert x.dtype == (torch.float32 if prec == HB_F32 else torch.float64)
        if y is None:
            y = torch.empty_like(x)
        assert x.is_cuda and x.is_contiguous() and x.numel() == self.n_global
        hb_apply_A(self.handle, prec, screen, lam, x.data_ptr(), y.data_ptr(), stream)
        return y

    def dot(self, a, b, stream=None):
        import torch
        prec = HB_F64 if a.dtype == torch.float64 else HB_F32
        return hb_dot(self.handle, prec, a.data_ptr(), b.data_ptr(), None, True, stream)

    def rhs(self, kind=0, seed=0, lam=0.0, stream=None):
        b = self.vec()
        hb_fill_rhs(self.handle, kind, seed, lam, b.data_ptr(), stream)
        return b

    def cg(self, b, x=None, lam=0.0, rtol=0.0, max_it=100, prec=HB_F64, screen=HB_SCREEN_IDENTITY,
           inner_rtol=1e-4, max_outer=30, precond=0, stream=None):
        if x is None:
            x = self.vec()
        opts = hb_cg_opts(prec, screen, lam, rtol, max_it, inner_rtol, max_outer, precond)
        res = hb_cg_solve(self.handle, opts, b.data_ptr(), x.data_ptr(), stream)
        return x, res

    def cg_begin(self, b, x, lam=0.0, rtol=0.0, max_it=100, prec=HB_F64, screen=HB_SCREEN_IDENTITY, precond=0,
                 stream=None):
        """Stepwise solve: r0 and the state (see hb_cg_begin); b and x must stay alive until cg_finish."""
        opts = hb_cg_opts(prec, screen, lam, rtol, max_it, 0.0, 0, precond)
        _check(lib().hb_cg_begin(self.handle, C.byref(opts), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                 _stream_ptr(stream)))

    def cg_iterate(self, count, stream=None):
        _check(lib().hb_cg_iterate(self.handle, count, _stream_ptr(stream)))

    def cg_finish(self, stream=None) -> hb_cg_result:
        res = hb_cg_result()
        st = lib().hb_cg_finish(self.handle, C.byref(res), _stream_ptr(stream))
        if st not in (HB_OK, HB_ERR_NOT_CONVERGED, HB_ERR_BREAKDOWN):
            _check(st)
        return res

    def diag_A(self, lam=0.0, screen=HB_SCREEN_IDENTITY, stream=None):
        import numpy as np
        out = np.zeros(self.n_global)
        _check(lib().hb_diag_A(self.handle, screen, lam, out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return out

    def l2g(self):
        import numpy as np
        out = np.zeros(self.n_local, dtype=np.int32)
        _check(lib().hb_mesh_copy_l2g(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out

    def geo(self):
        import numpy as np
        out = np.zeros(7 * self.n_local, dtype=np.float64)
        _check(lib().hb_mesh_copy_geo(self.handle, out.ctypes.data_as(C.c_void_p)))
        return out


# ---------------------------------------------------------------- partitioned operator

def hb_part_plan(l2g, dims, N, n_global, grid, seed=0):
    """Host-only partition plan of a box mesh from its node map (numpy int32,
    E*(N+1)^3 values). Returns (perm, n_shared, exchange_values, per-rank
    counts as an int64 array [P][8]: n_owned, offset, n_halo, n_send,
    n_elem_interior1, n_elem_halo, n_elem_interior2, n_owned_shared)."""
    import numpy as np
    l2g = np.ascontiguousarray(l2g, dtype=np.int32)
    P = grid[0] * grid[1] * grid[2]
    perm = np.empty(n_global, dtype=np.int32)
    counts = np.zeros(2 + 8 * P, dtype=np.int64)
    _check(lib().hb_part_plan(l2g.ctypes.data_as(C.c_void_p), dims[0], dims[1], dims[2], N, n_global, grid[0],
                              grid[1], grid[2], seed, perm.ctypes.data_as(C.c_void_p),
                              counts.ctypes.data_as(C.c_void_p)))
    return perm, int(counts[0]), int(counts[1]), counts[2:].reshape(P, 8)


class Part:
    """Owns one hb_part: the operator split over px*py*pz virtual ranks of
    `mesh` (which must stay open). Vectors are FP64 torch CUDA tensors in
    partition order; `perm[i]` is the mesh's global id of entry i."""

    def __init__(self, mesh, px, py, pz, seed=0, stream=None):
        import numpy as np
        self.mesh = mesh
        h = C.c_void_p()
        _check(lib().hb_part_create(mesh.handle, px, py, pz, seed, _stream_ptr(stream), C.byref(h)))
        self.handle = h
        info = hb_part_info_t()
        _check(lib().hb_part_info(h, C.byref(info)))
        self.info = info
        self.n_ranks = info.n_ranks
        self.n_global = info.n_global
        self.perm = np.empty(self.n_global, dtype=np.int32)
        _check(lib().hb_part_copy_perm(h, self.perm.ctypes.data_as(C.c_void_p)))

    def rank_info(self, rank) -> hb_part_rank_info_t:
        out = hb_part_rank_info_t()
        _check(lib().hb_part_rank_info(self.handle, rank, C.byref(out)))
        return out

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().hb_part_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self):
        import torch
        return torch.zeros(self.n_global, dtype=torch.float64, device="cuda")

    def apply_A(self, x, y=None, lam=0.0, screen=HB_SCREEN_IDENTITY, stream=None):
        import torch
        assert x.is_cuda and x.dtype == torch.float64 and x.numel() == self.n_global
        if y is None:
            y = torch.empty_like(x)
        _check(lib().hb_part_apply_A(self.handle, screen, lam, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                     _stream_ptr(stream)))
        return y

    def halo_exchange(self, x, rank=-1, stream=None):
        """Fills every rank's halo buffer from x; returns rank `rank`'s buffer
        as a numpy array (None for rank < 0)."""
        import numpy as np
        if rank < 0:
            _check(lib().hb_part_halo_exchange(self.handle, C.c_void_p(x.data_ptr()), -1, None,
                                               _stream_ptr(stream)))
            return None
        out = np.empty(self.rank_info(rank).n_halo, dtype=np.float64)
        _check(lib().hb_part_halo_exchange(self.handle, C.c_void_p(x.data_ptr()), rank,
                                           out.ctypes.data_as(C.c_void_p), _stream_ptr(stream)))
        return out

    def cg(self, b, x=None, lam=0.0, rtol=0.0, max_it=100, screen=HB_SCREEN_IDENTITY, stream=None):
        if x is None:
            x = self.vec()
        opts = hb_cg_opts(HB_F64, screen, lam, rtol, max_it, 0.0, 0, 0)
        res = hb_cg_result()
        st = lib().hb_part_cg_solve(self.handle, C.byref(opts), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                    C.byref(res), _stream_ptr(stream))
        if st not in (HB_OK, HB_ERR_NOT_CONVERGED, HB_ERR_BREAKDOWN):
            _check(st)
        return x, res


# ---------------------------------------------------------------- scattered storage

class Scat:
    """Owns one hb_scat: NekBone's scattered (n_local) vectors of `mesh`
    (which must stay open). Vectors are FP64 torch CUDA tensors of n_local."""

    def __init__(self, mesh, stream=None):
        self.mesh = mesh
        h = C.c_void_p()
        _check(lib().hb_scat_create(mesh.handle, _stream_ptr(stream), C.byref(h)))
        self.handle = h
        self.n_local = mesh.n_local

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().hb_scat_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def vec(self):
        import torch
        return torch.zeros(self.n_local, dtype=torch.float64, device="cuda")

    def scatter(self, xG, xL=None, stream=None):
        if xL is None:
            xL = self.vec()
        _check(lib().hb_scat_scatter(self.handle, C.c_void_p(xG.data_ptr()), C.c_void_p(xL.data_ptr()),
                                     _stream_ptr(stream)))
        return xL

    def apply_A(self, xL, yL=None, lam=0.0, screen=HB_SCREEN_IDENTITY, stream=None):
        import torch
        assert xL.is_cuda and xL.dtype == torch.float64 and xL.numel() == self.n_local
        if yL is None:
            yL = torch.empty_like(xL)
        _check(lib().hb_scat_apply_A(self.handle, screen, lam, C.c_void_p(xL.data_ptr()), C.c_void_p(yL.data_ptr()),
                                     _stream_ptr(stream)))
        return yL

    def dot(self, a, b, stream=None) -> float:
        out = C.c_double()
        _check(lib().hb_scat_dot(self.handle, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), C.byref(out),
                                 _stream_ptr(stream)))
        return out.value

    def cg(self, bL, xL=None, lam=0.0, rtol=0.0, max_it=100, screen=HB_SCREEN_IDENTITY, stream=None):
        if xL is None:
            xL = self.vec()
        opts = hb_cg_opts(HB_F64, screen, lam, rtol, max_it, 0.0, 0, 0)
        res = hb_cg_result()
        st = lib().hb_scat_cg_solve(self.handle, C.byref(opts), C.c_void_p(bL.data_ptr()),
                                    C.c_void_p(xL.data_ptr()), C.byref(res), _stream_ptr(stream))
        if st not in (HB_OK, HB_ERR_NOT_CONVERGED, HB_ERR_BREAKDOWN):
            _check(st)
        return xL, res


# ---------------------------------------------------------------- server

class Server:
    """Owns an hb_server (continuous-batching CG server on the current GPU)."""

    def __init__(self, mem_budget_bytes, max_slots=16, iters_per_launch=8):
        o = hb_server_opts(int(mem_budget_bytes), max_slots, iters_per_launch)
        h = C.c_void_p()
        _check(lib().hb_server_create(C.byref(o), C.byref(h)))
        self.handle = h

    def submit(self, ex, ey, ez, N, perturb=0.1, seed=0, rhs_seed=0, lam=0.1, rtol=1e-8, max_it=100000,
               inner_rtol=1e-4, max_outer=30, screen=HB_SCREEN_IDENTITY, faces=ALL_FACES, keep_x=False) -> int:
        d = hb_mesh_desc(ex, ey, ez, N, perturb, seed, faces, 1)
        o = hb_cg_opts(HB_MIXED, screen, lam, rtol, max_it, inner_rtol, max_outer, 0)
        t = C.c_int64(0)
        _check(lib().hb_server_submit(self.handle, C.byref(d), C.byref(o), rhs_seed, 1 if keep_x else 0,
                                      C.byref(t)))
        return t.value

    def poll(self, ticket, n_global=None):
        """None while queued or running; else (hb_cg_result, x or None)."""
        import numpy as np
        res = hb_cg_result()
        ng = C.c_int64(0)
        x = np.zeros(n_global, dtype=np.float64) if n_global else None
        st = lib().hb_server_poll(self.handle, ticket, C.byref(res), C.byref(ng),
                                  x.ctypes.data_as(C.c_void_p) if x is not None else None)
        if st == HB_ERR_BUSY:
            return None
        _check(st)
        if res.status != HB_OK:
            self.last_failure = lib().hb_last_error().decode(errors="replace")
        return res, x

    def wait(self, ticket, n_global=None, timeout=600.0, interval=0.0005):
        import time
        t0 = time.time()
        while True:
            r = self.poll(ticket, n_global)
            if r is not None:
                return r
            if time.time() - t0 > timeout:
                raise TimeoutError(f"ticket {ticket} not done after {timeout} s")
            time.sleep(interval)

    def inject_round_error(self) -> None:
        """Test hook: the next round fails as if its launch had failed."""
        _check(lib().hb_server_inject_round_error(self.handle))

    def stats(self) -> hb_server_stats_t:
        st = hb_server_stats_t()
        _check(lib().hb_server_stats(self.handle, C.byref(st)))
        return st

    def close(self):
        if getattr(self, "handle", None):
            _check(lib().hb_server_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def hb_tc_selftest(mode, A, B):
    """D = A B^T on the tensor cores (see the C header); A 128x48, B 48x48
    float32 numpy arrays. Returns (D, status)."""
    import numpy as np
    A = np.ascontiguousarray(A, dtype=np.float32)
    B = np.ascontiguousarray(B, dtype=np.float32)
    D = np.zeros((128, 48), dtype=np.float32)
    st = C.c_int(-1)
    _check(lib().hb_tc_selftest(mode, A.ctypes.data_as(C.c_void_p), B.ctypes.data_as(C.c_void_p),
                                D.ctypes.data_as(C.c_void_p), C.byref(st)))
    return D, st.value
