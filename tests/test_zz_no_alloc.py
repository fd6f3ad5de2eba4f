"""hb_dot_noalloc: the dot product for callers that may not allocate device
memory (their own allocator holds the device, or their loop cannot take the
synchronisation an allocation may cause). It keeps its scratch in a static
array inside the library instead of the mesh workspace hb_dot uses.

Checked through the C ABI against hb_dot, on two calls in a row, within the
dot-product bar of the other tests (1e-14 of sum |a_i b_i| for FP64, 1e-13
for FP32). This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2202_12477_gb300 import hb, inputs  # noqa: E402

MAX_N = 16384 * 1024


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


def _noalloc(prec, a, b, n, out_dev=None):
    out = C.c_double(float("nan"))
    st = hb.lib().hb_dot_noalloc(prec, C.c_void_p(a.data_ptr()), C.c_void_p(b.data_ptr()), n,
                                 C.c_void_p(out_dev.data_ptr() if out_dev is not None else 0), C.byref(out),
                                 C.c_void_p(torch.cuda.current_stream().cuda_stream))
    return st, out.value


@pytest.mark.parametrize("dims,N", [((8, 8, 8), 7), ((30, 30, 30), 7)])
@pytest.mark.parametrize("dtype,prec,bar", [(torch.float64, hb.HB_F64, 1e-14), (torch.float32, hb.HB_F32, 1e-13)])
def test_noalloc_dot_matches_hb_dot_twice(dims, N, dtype, prec, bar):
    m = hb.Mesh(*dims, N, fp32=False)
    n = m.n_global
    vecs = [torch.from_numpy(inputs.random_vector(n, s, "normal")).to("cuda", dtype) for s in (11, 12, 13, 14)]
    pairs = [(vecs[0], vecs[1]), (vecs[2], vecs[3])]
    dev_out = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    for call, (a, b) in enumerate(pairs):
        ref = hb.hb_dot(m.handle, prec, a.data_ptr(), b.data_ptr())
        st, got = _noalloc(prec, a, b, n, out_dev=dev_out if call == 1 else None)
        assert st == hb.HB_OK, hb.lib().hb_last_error()
        scale = float((a.double() * b.double()).abs().sum())
        assert abs(got - ref) <= bar * scale, (call, got, ref)
        if n <= 1216 * 1024:
            assert got == ref  # same grid as hb_dot: bitwise equal
        if call == 1:
            assert float(dev_out.item()) == got
    m.close()


def test_noalloc_dot_allocates_no_device_memory():
    """The property the entry point exists for: after a first call (which
    takes the scratch array's address), further calls leave the device's
    free memory unchanged."""
    n = 1 << 20
    a = torch.from_numpy(inputs.random_vector(n, 21, "normal")).cuda()
    b = torch.from_numpy(inputs.random_vector(n, 22, "normal")).cuda()
    st, first = _noalloc(hb.HB_F64, a, b, n)
    assert st == hb.HB_OK, hb.lib().hb_last_error()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(8):
        st, v = _noalloc(hb.HB_F64, a, b, n)
        assert st == hb.HB_OK and v == first
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_noalloc_dot_rejects_lengths_beyond_its_scratch():
    a = torch.zeros(16, dtype=torch.float64, device="cuda")
    st, _ = _noalloc(hb.HB_F64, a, a, MAX_N + 1)
    assert st == hb.HB_ERR_ARG
    assert b"maximum" in hb.lib().hb_last_error()
    st, v = _noalloc(hb.HB_F64, a, a, 0)
    assert st == hb.HB_OK and v == 0.0
