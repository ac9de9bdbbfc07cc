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
    """Calls in a row with different shapes, the largest documented one
    included (p + ones = 65, q = 64: every scratch slot up to the arrival
    counter), each checked entry by entry against the FP64 host product
    [1/n * 1 | A]^T B with a bound scaled by |A|^T |B| (a dropped or doubled
    row tile, or a wrong column-mean row, exceeds it by orders of magnitude),
    and against the handle-based lap_gram."""
    n = 50_000 + 37  # several tiles and a ragged tail
    gph = G.path_graph(n)  # lap_gram only needs the handle's row layout
    H = pkg.Graph(gph)
    rel = 1e-12 if dt == torch.float64 else 1e-5
    cases = [(12, 9, 1), (40, 20, 0), (64, 64, 1), (30, 64, 0), (0, 5, 1)]
    for i, (p, q, ones) in enumerate(cases):
        npdt = np.float64 if dt == torch.float64 else np.float32
        A64 = G.random_block(n, p, 10 + i).astype(npdt).astype(np.float64)
        B64 = G.random_block(n, q, 20 + i).astype(npdt).astype(np.float64)
        A = torch.from_numpy(A64).to(dt).cuda() if p else None
        B = torch.from_numpy(B64).to(dt).cuda()
        got = _noalloc(pkg, A, B, ones).cpu().numpy()
        ref = A64.T @ B64
        bound = np.abs(A64).T @ np.abs(B64)
        if ones:
            ref = np.vstack([B64.mean(axis=0, keepdims=True), ref])
            bound = np.vstack([np.abs(B64).mean(axis=0, keepdims=True), bound])
        assert got.shape == ref.shape
        assert np.all(np.abs(got - ref) <= rel * bound), np.max(np.abs(got - ref) / bound)
        if p:
            lg = H.gram(A, B, ones=bool(ones)).cpu().numpy()[0]
            assert np.all(np.abs(got - lg) <= 2 * rel * bound)
    H.close()


def test_noalloc_rejects_oversize(pkg):
    B = torch.zeros((100, 65), dtype=torch.float64, device="cuda")
    Gm = torch.zeros((1, 65), dtype=torch.float64, device="cuda")
    st = pkg.lib().lap_gram_noalloc(100, pkg.LAP_F64, None, 0, 0, ctypes.c_void_p(B.data_ptr()), 65, 65, 1,
                                    ctypes.c_void_p(Gm.data_ptr()), None)
    assert st == pkg.LAP_EINVAL
    assert b"q <= 64" in pkg.lib().lap_last_error()
