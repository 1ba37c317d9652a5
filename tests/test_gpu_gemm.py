"""The contraction kernels on their own (mps_zgemm_mixed_dev), against numpy in FP64.

FP64 kernel: 1e-13 relative.  Split-TF32 kernels (the mma.sync one and the tcgen05 one with
tensor-memory accumulators): each real operand is split into two TF32 parts and products are
accumulated in FP32, so an element of C is accurate to about 1e-6 of sum_k |A_ik| |B_kj|.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    import torch
    assert torch.cuda.is_available()
    from paper_2211_07983_gb300 import build
    build.build()
    import paper_2211_07983_gb300 as M
    return M


def _op(X, op):
    return {"N": X, "T": X.T, "H": X.conj().T, "C": X.conj()}[op]


@pytest.mark.parametrize("engine", ["tcgen05", "mma_sync", "fp64"])
@pytest.mark.parametrize("m,n,k,opA,opB", [(128, 128, 16, "N", "N"), (128, 128, 256, "N", "N"),
                                           (256, 512, 256, "N", "N"), (200, 130, 77, "H", "N"),
                                           (64, 256, 512, "H", "N"), (256, 256, 512, "N", "T"),
                                           (96, 300, 40, "C", "H"), (8, 8, 8, "N", "N"), (130, 1, 5, "T", "C")])
def test_complex_gemm_kernels_against_numpy(M, engine, m, n, k, opA, opB):
    import torch
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    shapeA = (m, k) if opA in ("N", "C") else (k, m)
    shapeB = (k, n) if opB in ("N", "C") else (n, k)
    A = rng.standard_normal(shapeA) + 1j * rng.standard_normal(shapeA)
    B = rng.standard_normal(shapeB) + 1j * rng.standard_normal(shapeB)
    ref = _op(A, opA) @ _op(B, opB)
    C = M.api.zgemm(torch.tensor(A, device="cuda"), torch.tensor(B, device="cuda"), opA, opB, engine).cpu().numpy()
    scale = np.abs(_op(A, opA)) @ np.abs(_op(B, opB))
    tol = 1e-13 if engine == "fp64" else 2e-6
    assert np.all(np.abs(C - ref) <= tol * scale + 1e-300)
