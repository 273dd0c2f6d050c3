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


def _forward(src, S, per, gather, levels=4, seed=3):
    import os
    from paper_1709_04703_gb300.guess import GuessNet
    old = os.environ.pop("PM_NN_GATHER", None)
    if gather:
        os.environ["PM_NN_GATHER"] = "1"
    try:
        net = GuessNet(levels=levels, seed=seed)
    finally:
        os.environ.pop("PM_NN_GATHER", None)
        if old is not None:
            os.environ["PM_NN_GATHER"] = old
    out = net.forward(src, periodic=per).cpu().numpy()
    net.close()
    return out


@pytest.mark.parametrize("S,B,per", [(32, 1, 0), (32, 2, 1), (40, 1, 0), (24, 1, 1),
                                     (64, 1, 0), (16, 2, 1)])
def test_staged_forward_matches_gathered(lib, S, B, per):
    """The staged-input convolution (tap-shifted operands of one shared
    block, k_conv.cu) against the gathered-tile one on the same network:
    the same convolutions, FP32 accumulation in another order, so the
    outputs agree to BF16 rounding of the activations (blocks of side 11,
    8 and 6 with partial blocks at the sample edge: 32, 40, 24 and 16 are
    not multiples of them)."""
    g = torch.Generator().manual_seed(S + B + per)
    src = torch.randn(B, S, S, S, generator=g).cuda()
    a = _forward(src, S, per, gather=False)
    b = _forward(src, S, per, gather=True)
    err = np.sqrt(((a - b) ** 2).sum() / (b**2).sum())
    assert err < 5e-3, err
