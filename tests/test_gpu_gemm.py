"""The tcgen05 BF16 GEMM against FP64 products of the same BF16 operands.

Bound per element: |D - D*| <= K 2^-24 (|A| |B|^T) (FP32 accumulation of exact
BF16 x BF16 products), plus half an ulp of BF16 for BF16 outputs."""
import ctypes

import numpy as np
import pytest

from oracle.mlp import bf16_round

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

from paper_2311_16728_b300 import _lib as L  # noqa: E402


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _gemm(A, B, *, bias=None, relu=0, mask=None, out="f32", transposed=False, colsum=None, valid=None, ksplit=1,
          atomic=0, pad=0):
    """pad: extra elements per row of the mask, the BF16 outputs and the
    transposed output (pad % 8 != 0 takes the epilogue's unvectorised paths)."""
    M, K = A.shape
    N = B.shape[0]
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    of = torch.zeros(M, N, device="cuda") if out == "f32" else None
    ob = torch.zeros(M, N + pad, dtype=torch.bfloat16, device="cuda") if out == "bf16" else None
    ot = torch.zeros(N, M + pad, dtype=torch.bfloat16, device="cuda") if transposed else None
    mk = None
    if mask is not None:
        mk = torch.zeros(M, N + pad, dtype=torch.bfloat16, device="cuda")
        mk[:, :N] = mask
    L.gsr_gemm_bf16(_p(A), K, _p(B), K, M, N, K, _p(bias), relu, _p(mk), N + pad, _p(ob), N + pad, _p(ot), M + pad,
                    _p(of), N, atomic, _p(colsum), M if valid is None else valid, ksplit, _p(status), st)
    torch.cuda.synchronize()
    assert int(status.item()) == 0
    return of, None if ob is None else ob[:, :N], None if ot is None else ot[:, :M]


def _operands(M, N, K, seed):
    rng = np.random.default_rng(seed)
    a = rng.standard_normal((M, K)).astype(np.float32)
    b = rng.standard_normal((N, K)).astype(np.float32)
    At = torch.tensor(a, device="cuda").to(torch.bfloat16)
    Bt = torch.tensor(b, device="cuda").to(torch.bfloat16)
    a64, b64 = bf16_round(a), bf16_round(b)
    return At, Bt, a64, b64


@pytest.mark.parametrize("M,N,K", [(128, 64, 64), (128, 128, 128), (256, 256, 320), (384, 64, 2368),
                                   (128, 2368, 256)])
def test_gemm_fp32_output(M, N, K):
    At, Bt, a64, b64 = _operands(M, N, K, seed=M + N + K)
    of, _, _ = _gemm(At, Bt)
    ref = a64 @ b64.T
    bound = K * 2.0 ** -24 * (np.abs(a64) @ np.abs(b64).T) + 1e-30
    err = np.abs(of.cpu().numpy() - ref)
    assert (err <= bound).all(), f"max err/bound {(err / bound).max():.3f}"


@pytest.mark.parametrize("pad", [0, 3])
def test_gemm_epilogue_bias_relu_bf16_transposed_colsum(pad):
    M, N, K = 256, 128, 192
    At, Bt, a64, b64 = _operands(M, N, K, seed=9)
    bias = torch.tensor(np.random.default_rng(10).standard_normal(N).astype(np.float32), device="cuda")
    colsum = torch.zeros(N, device="cuda")
    _, ob, ot = _gemm(At, Bt, bias=bias, relu=1, out="bf16", transposed=True, colsum=colsum, valid=200, pad=pad)
    ref = np.maximum(a64 @ b64.T + bias.cpu().numpy().astype(np.float64), 0)
    bound = K * 2.0 ** -24 * (np.abs(a64) @ np.abs(b64).T) + np.abs(bias.cpu().numpy())[None] * 2 ** -24
    got = ob.float().cpu().numpy()
    # bf16 keeps 8 significant bits (unit roundoff 2^-8), so with |g - r| <= bound:
    # |bf16(g) - bf16(r)| <= 2^-8 |g| + |g - r| + 2^-8 |r| <= bound (1 + 2^-8) + 2^-7 |r|
    # (one bf16 ulp: an FP32 sum next to a rounding midpoint may round the other way)
    assert (np.abs(got - bf16_round(ref)) <= bound * (1 + 2 ** -8) + np.abs(ref) * 2 ** -7 + 1e-30).all()
    assert torch.equal(ot, ob.t().contiguous())
    np.testing.assert_allclose(colsum.cpu().numpy(), ref[:200].sum(0), rtol=1e-5, atol=1e-3)


@pytest.mark.parametrize("pad", [0, 3])
def test_gemm_relu_mask_and_split_k(pad):
    M, N, K = 128, 64, 1024
    At, Bt, a64, b64 = _operands(M, N, K, seed=5)
    mask = torch.randn(M, N, device="cuda").to(torch.bfloat16)
    of, _, _ = _gemm(At, Bt, mask=mask, pad=pad)
    ref = (a64 @ b64.T) * (mask.float().cpu().numpy() > 0)
    bound = K * 2.0 ** -24 * (np.abs(a64) @ np.abs(b64).T) + 1e-30
    assert (np.abs(of.cpu().numpy() - ref) <= bound).all()
    of2, _, _ = _gemm(At, Bt, ksplit=4, atomic=1)
    ref2 = a64 @ b64.T
    assert (np.abs(of2.cpu().numpy() - ref2) <= 2 * bound).all()
