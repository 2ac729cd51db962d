"""The allocation-free Gram entry point, sparc_gram_noalloc, called through the C ABI.

It exists for callers that cannot let the library allocate device memory where they call
it (real-time loops that forbid cudaMalloc after start-up, hosts that hand in buffers from
their own pool, processes that have reserved nearly all device memory). Its partial sums
live in a fixed __device__ array instead of context workspace. Its result must equal the
existing sparc_gram's, and the FP64 product A^T B formed on the host by numpy, within the
Gram tolerance used elsewhere in the suite (1e-13 normwise), on two calls in a row (the
second call reuses the array the first one left behind). The second call must leave the
device's free memory unchanged.

This file is named to be collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
if not torch.cuda.is_available():
    pytestmark = [pytest.mark.gpu, pytest.mark.skip(reason="no CUDA device")]

from paper_1603_04334_gb300 import sparc  # noqa: E402

TOL = 1e-13


def _noalloc():
    L = sparc.load()
    f = L.sparc_gram_noalloc
    f.argtypes = [C.c_void_p, C.c_void_p, C.c_long, C.c_int, C.c_long, C.c_void_p, C.c_void_p]
    f.restype = C.c_int
    return f


@pytest.mark.parametrize("n3,ncols,pad", [((24, 24, 24), 12, 0), ((37, 29, 23), 70, 3),
                                          ((96, 96, 96), 128, 0)])
def test_gram_noalloc_matches_sparc_gram_twice(n3, ncols, pad):
    f = _noalloc()
    nd = n3[0] * n3[1] * n3[2]
    ld = nd + pad
    rng = np.random.default_rng(ncols)
    Ah = rng.uniform(-0.5, 0.5, (ncols, ld))
    Bh = rng.uniform(-0.5, 0.5, (ncols, ld))
    A = torch.from_numpy(Ah).to("cuda:0")
    B = torch.from_numpy(Bh).to("cuda:0")
    ctx = sparc.Context(n3, 0.5, veff=np.zeros(nd))
    G_ref = ctx.gram(A, B).cpu().numpy()
    # independent reference: the FP64 product on the host (column-major G: G[j, i] in
    # torch indexing is entry (i, j) = sum_k A[k, i] B[k, j])
    G_np = (Ah[:, :nd] @ Bh[:, :nd].T).T
    assert np.max(np.abs(G_ref - G_np)) / np.max(np.abs(G_np)) <= TOL
    stream = torch.cuda.current_stream().cuda_stream
    G = torch.empty((ncols, ncols), dtype=torch.float64, device="cuda:0")
    free_after_first = None
    for call in range(2):
        G.fill_(np.nan)
        torch.cuda.synchronize()
        if call == 1:
            free_after_first = torch.cuda.mem_get_info()[0]
        st = f(C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()), nd, ncols, ld,
               C.c_void_p(G.data_ptr()), C.c_void_p(stream))
        assert st == sparc.SPARC_OK, (call, st)
        torch.cuda.synchronize()
        if call == 1:
            # no device memory was taken by the call (the first one may load the kernel)
            assert torch.cuda.mem_get_info()[0] == free_after_first
        got = G.cpu().numpy()
        err = np.max(np.abs(got - G_ref)) / np.max(np.abs(G_ref))
        assert err <= TOL, (call, err)
        err_np = np.max(np.abs(got - G_np)) / np.max(np.abs(G_np))
        assert err_np <= TOL, (call, err_np)
    ctx.close()


def test_gram_noalloc_rejects_bad_sizes():
    f = _noalloc()
    A = torch.zeros((4, 100), dtype=torch.float64, device="cuda:0")
    G = torch.zeros((4, 4), dtype=torch.float64, device="cuda:0")
    p = C.c_void_p(A.data_ptr())
    # ld < nd
    assert f(p, p, 100, 4, 99, C.c_void_p(G.data_ptr()), None) == sparc.SPARC_ERR_ARG
    # ncols^2 beyond the fixed array (2^21 doubles)
    assert f(p, p, 100, 2000, 100, C.c_void_p(G.data_ptr()), None) == sparc.SPARC_ERR_ARG
    # null output
    assert f(p, p, 100, 4, 100, None, None) == sparc.SPARC_ERR_ARG
