"""mps_svd_noalloc: the gate SVD for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: embedders whose device memory belongs to another allocator
(or to a pool sized once at start-up), and latency-critical loops that cannot afford the device
synchronisation an allocation can imply.  The no-allocation entry point serves them from a
fixed scratch array inside the library.  This test calls it through the C ABI on two different
matrices in a row and checks each result against the allocating entry point mps_svd_dev.
It lives in its own file, collected last.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call_noalloc(lib, A_dev, m, n, D, eps, torch):
    K = min(m, n)
    s = torch.zeros(K, dtype=torch.float64, device="cuda")
    V = torch.zeros(n * K * 2, dtype=torch.float64, device="cuda")
    W = torch.zeros(m * K * 2, dtype=torch.float64, device="cuda")
    k = torch.zeros(1, dtype=torch.int32, device="cuda")
    fn = lib.mps_svd_noalloc
    fn.restype = ctypes.c_int32
    fn.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_int32, ctypes.c_double,
                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]
    code = fn(m, n, A_dev.data_ptr(), D, eps, s.data_ptr(), V.data_ptr(), W.data_ptr(), k.data_ptr(), None)
    return code, s.cpu().numpy(), V.cpu().numpy().view(np.complex128).reshape(n, K), \
        W.cpu().numpy().view(np.complex128).reshape(m, K), int(k.item())


def test_no_alloc_svd_matches_allocating_entry_point_twice_in_a_row():
    torch = pytest.importorskip("torch")
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import _lib, build
    build.build()
    import paper_2211_07983_gb300 as M
    lib = _lib.load()
    rng = np.random.default_rng(2211)
    for (m, n, r) in [(64, 64, 40), (32, 128, 20)]:        # two different calls, one after the other
        A = (rng.standard_normal((m, r)) + 1j * rng.standard_normal((m, r))) @ (
            rng.standard_normal((r, n)) + 1j * rng.standard_normal((r, n)))
        s_ref, V_ref, W_ref, k_ref = M.svd(A, 64, 1e-12)
        A_dev = torch.tensor(np.ascontiguousarray(A).view(np.float64), device="cuda")
        code, s, V, W, k = _call_noalloc(lib, A_dev, m, n, 64, 1e-12, torch)
        assert code == 0, lib.mps_last_error()
        assert k == k_ref == r
        tol = 1e-12 * s_ref[0]
        assert np.abs(s - s_ref).max() <= tol
        assert np.abs(V[:, :r] - V_ref[:, :r]).max() <= 1e-12
        assert np.abs(W - W_ref).max() <= tol


def test_no_alloc_svd_rejects_sizes_beyond_its_scratch():
    torch = pytest.importorskip("torch")
    from paper_2211_07983_gb300 import _lib
    lib = _lib.load()
    A_dev = torch.zeros(256 * 256 * 2, dtype=torch.float64, device="cuda")
    code, *_ = _call_noalloc(lib, A_dev, 256, 256, 64, 1e-12, torch)
    assert code == 1                                      # MPS_EINVAL: beyond the fixed maximum
