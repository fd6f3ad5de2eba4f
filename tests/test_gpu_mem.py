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


def test_meshes_built_concurrently_from_two_threads():
    # two host threads build meshes of different degrees at the same time, as
    # the server's builders do; each operator matches a mesh built alone
    import threading

    cases = [(5, 4, 3, 3), (4, 3, 3, 11), (3, 3, 2, 7), (6, 2, 2, 9)]
    ref = {}
    for c in cases:
        m = hb.Mesh(*c, perturb=0.1, seed=1, fp32=True)
        x = torch.from_numpy(inputs.random_vector(m.n_global, seed=3)).cuda()
        ref[c] = (x, m.apply_A(x, lam=0.1).cpu().numpy())
        m.close()
    errors = []

    def build(order):
        try:
            s = torch.cuda.Stream()
            for _ in range(6):
                for c in order:
                    with torch.cuda.stream(s):
                        m = hb.Mesh(*c, perturb=0.1, seed=1, fp32=True)
                        y = m.apply_A(ref[c][0], lam=0.1)
                    s.synchronize()
                    if not np.array_equal(y.cpu().numpy(), ref[c][1]):
                        errors.append(f"mismatch {c}")
                    m.close()
        except Exception as e:  # noqa: BLE001
            errors.append(repr(e))

    ts = [threading.Thread(target=build, args=(cases,)), threading.Thread(target=build, args=(cases[::-1],))]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    assert not errors, errors
