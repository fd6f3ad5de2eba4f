"""Mesh memory: stream-ordered arrays from the library's pool, through the C ABI.

Checks: repeated create/destroy of a mesh reuses the pool's memory (the
device's free memory does not shrink cycle after cycle); a mesh built on one
stream is ready for work on another as soon as hb_mesh_create returns; the
operator of a rebuilt mesh is bitwise the same as the first one's.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

from paper_2202_12477_gb300 import hb, inputs  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    hb.lib()


def test_create_destroy_cycles_do_not_grow_device_memory():
    dims = (12, 12, 10, 7)
    m = hb.Mesh(*dims, perturb=0.1, seed=0, fp32=True)
    m.close()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for i in range(20):
        m = hb.Mesh(*dims, perturb=0.1, seed=i, fp32=True)
        m.close()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 >= free0 - (64 << 20), (free0, free1)


def test_mesh_from_a_side_stream_is_ready_on_another():
    side = torch.cuda.Stream()
    x = None
    ys = []
    for rep in range(2):
        with torch.cuda.stream(side):
            m = hb.Mesh(6, 5, 4, 7, perturb=0.15, seed=3, fp32=True)
        if x is None:
            x = torch.from_numpy(inputs.random_vector(m.n_global, seed=2)).cuda()
        # straight onto the default stream, no wait on the side stream
        ys.append(m.apply_A(x, lam=0.1).cpu().numpy())
        m.close()
    assert np.array_equal(ys[0], ys[1])
