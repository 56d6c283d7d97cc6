"""godec_mul_ZB_noalloc against godec_mul_ZB.

The no-allocation entry point exists for callers that cannot allocate device
memory while they run (for example an application that reserves all GPU memory
at start-up and forbids later allocations).  Its split-K scratch is a fixed
array inside the library, so two calls in a row must still give the same
product as the allocating entry point, whatever the first call left behind.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _noalloc(lib):
    f = lib.godec_mul_ZB_noalloc
    f.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64, ctypes.c_int64, ctypes.c_void_p,
                  ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p]
    f.restype = ctypes.c_int
    return f


def test_noalloc_product_matches_allocating_one_on_two_calls():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    lib = G.library()
    f = _noalloc(lib)
    stream = torch.cuda.current_stream().cuda_stream
    g = np.random.default_rng(2024)
    # a larger call first, then a smaller one that reuses the same scratch
    for (m, n, r) in [(3000, 2001, 50), (700, 513, 7)]:
        ldz = (n + 3) // 4 * 4
        Zh = np.zeros((m, ldz), np.float32)
        Zh[:, :n] = g.standard_normal((m, n))
        Bh = g.standard_normal((n, r)).astype(np.float32)
        Z = torch.from_numpy(Zh).cuda()
        B = torch.from_numpy(Bh).cuda()
        ref = G.mul_ZB(Z[:, :n], B)
        Y = torch.full((m, r), float("nan"), device="cuda")
        st = f(Z.data_ptr(), m, n, ldz, B.data_ptr(), r, Y.data_ptr(), stream)
        assert st == 0, lib.godec_last_error(None)
        torch.cuda.synchronize()
        Yn, Rn = Y.cpu().double().numpy(), ref.cpu().double().numpy()
        assert np.isfinite(Yn).all()
        assert np.linalg.norm(Yn - Rn) <= 1e-5 * np.linalg.norm(Rn)
        exact = Zh[:, :n].astype(np.float64) @ Bh.astype(np.float64)
        assert np.linalg.norm(Yn - exact) <= 1e-5 * np.linalg.norm(exact)


def test_noalloc_rejects_problems_above_its_scratch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_1309_0302_gb300 as G
    lib = G.library()
    f = _noalloc(lib)
    m, n, r = 200000, 8, 64                      # partial products alone exceed 32 MiB
    Z = torch.zeros((m, n), device="cuda")
    B = torch.zeros((n, r), device="cuda")
    Y = torch.zeros((m, r), device="cuda")
    st = f(Z.data_ptr(), m, n, n, B.data_ptr(), r, Y.data_ptr(), torch.cuda.current_stream().cuda_stream)
    assert st == 7
    assert b"scratch" in lib.godec_last_error(None)
