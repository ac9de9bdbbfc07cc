"""The allocation-free Gram product (lap_gram_noalloc) against lap_gram.

lap_gram_noalloc is for callers that may not allocate device memory (a
plug-in inside a framework that owns all device memory, or a latency-critical
caller that cannot afford cudaMalloc's synchronisation).  Its scratch is a
fixed device array shared by all calls, so this test calls it twice in a row
with different shapes and checks each result against the handle-based
lap_gram on the same inputs.  It lives in a file of its own, named to be
collected last, and must pass both alone and after the other tests."""
import ctypes

import numpy as np
import pytest

import graphgen as G

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    import paper_1311_1695_gb300 as p
    from paper_1311_1695_gb300 import build
    build.build()
    return p


def _noalloc(pkg, A, B, ones):
    n, q = B.shape
    p = 0 if A is None else A.shape[1]
    Gm = torch.zeros((p + ones, q), dtype=torch.float64, device="cuda")
    dtype = pkg.LAP_F64 if B.dtype == torch.float64 else pkg.LAP_F32
    pa = None if A is None else ctypes.c_void_p(A.data_ptr())
    st = pkg.lib().lap_gram_noalloc(n, dtype, pa, 0 if A is None else A.stride(0), p, ctypes.c_void_p(B.data_ptr()),
                                    B.stride(0), q, ones, ctypes.c_void_p(Gm.data_ptr()),
                                    ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert st == 0, pkg.lib().lap_last_error()
    return Gm


@pytest.mark.parametrize("dt", [torch.float64, torch.float32])
def test_noalloc_matches_lap_gram_twice(pkg, dt):
    n = 50_000 + 37  # several tiles and a ragged tail
    gph = G.path_graph(n)  # lap_gram only needs the handle's row layout
    H = pkg.Graph(gph)
    cases = [(12, 9, 1), (40, 20, 0)]  # two calls in a row, different shapes
    for i, (p, q, ones) in enumerate(cases):
        A = torch.from_numpy(G.random_block(n, p, 10 + i)).to(dt).cuda()
        B = torch.from_numpy(G.random_block(n, q, 20 + i)).to(dt).cuda()
        got = _noalloc(pkg, A, B, ones).cpu().numpy()
        ref = H.gram(A, B, ones=bool(ones)).cpu().numpy()[0]
        eps = np.finfo(np.float64 if dt == torch.float64 else np.float32).eps
        tol = (64 if dt == torch.float64 else 64 * 32) * eps * n
        assert got.shape == ref.shape
        assert np.abs(got - ref).max() <= tol, np.abs(got - ref).max()
    H.close()


def test_noalloc_rejects_oversize(pkg):
    B = torch.zeros((100, 65), dtype=torch.float64, device="cuda")
    Gm = torch.zeros((1, 65), dtype=torch.float64, device="cuda")
    st = pkg.lib().lap_gram_noalloc(100, pkg.LAP_F64, None, 0, 0, ctypes.c_void_p(B.data_ptr()), 65, 65, 1,
                                    ctypes.c_void_p(Gm.data_ptr()), None)
    assert st == pkg.LAP_EINVAL
    assert b"q <= 64" in pkg.lib().lap_last_error()
