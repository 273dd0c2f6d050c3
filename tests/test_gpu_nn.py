"""Tensor-core (tcgen05) building blocks of the learned initial guess against
FP64 references computed from the same BF16-rounded operands."""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_1709_04703_gb300 import _lib as L  # noqa: E402


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1709_04703_gb300 import build
    build.build()
    return L.load()


def _p(t):
    return C.c_void_p(t.data_ptr())


@pytest.mark.parametrize("M,N,K", [(128, 16, 64), (256, 64, 192), (384, 32, 640),
                                   (128, 128, 128)])
def test_tc_gemm_matches_fp64(lib, M, N, K):
    g = torch.Generator().manual_seed(M + N + K)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16).cuda()
    B = torch.randn(N, K, generator=g).to(torch.bfloat16).cuda()
    Cm = torch.full((M, N), float("nan"), dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    code = lib.pm_nn_gemm_bf16(_p(A), _p(B), _p(Cm), M, N, K, None)
    assert code == L.PM_OK, lib.pm_last_error(None)
    ref = A.double().cpu().numpy() @ B.double().cpu().numpy().T
    got = Cm.cpu().numpy().astype(np.float64)
    # FP32 accumulation of K products of BF16 values
    tol = 1e-6 * np.sqrt(K) * np.abs(A.double().cpu().numpy()).max() * \
        np.abs(B.double().cpu().numpy()).max() * 8
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol)
