"""The FP64 matrix product of the incremental SVD (Sec. 4.2 projections
W^T U and updates U - W L) through st_gemm_f64, on both arithmetic paths:
FP64 SIMT and the BF16 tensor-core path with exact 8-digit operand splits.

Pins: integer-valued operands whose products and sums are exact in FP64 must
come out bit-exact (the splitting is exact for them and every digit sum is an
exact FP32 integer); random operands with rows scaled over 2^+-29 must agree
with numpy's FP64 product within 1e-14 of |alpha| |A| |B| + |beta| |C|
elementwise (an FP64 GEMM's own rounding is ~K 2^-53 of that bound; a dropped
digit diagonal would show at 2^-35)."""
import numpy as np
import pytest

from gpu_util import torch_mod

pytestmark = pytest.mark.gpu


def _model(mode):
    import paper_1910_01260_gb300 as st
    torch = torch_mod()
    # a 1 x 1 operator: st_gemm_f64 needs only the model's stream and options
    return st.Model([0, 1], [0], [1.0], st.options(fp64_gemm=mode), stream=torch.cuda.current_stream().cuda_stream)


def _dev(X):
    """Column-major device copy of X with leading dimension X.shape[0]."""
    torch = torch_mod()
    return torch.tensor(np.ascontiguousarray(X.T), dtype=torch.float64, device="cuda")


def _host(t, rows):
    return t.cpu().numpy().T[:rows].copy()


def _gemm(m, ta, tb, A, B, alpha=1.0, beta=0.0, C0=None):
    """C = alpha op(A) op(B) + beta C0 through the C ABI; A, B host arrays as stored."""
    torch = torch_mod()
    M = A.shape[1] if ta else A.shape[0]
    K = A.shape[0] if ta else A.shape[1]
    N = B.shape[0] if tb else B.shape[1]
    dA, dB = _dev(A), _dev(B)
    C = _dev(C0 if C0 is not None else np.zeros((M, N)))
    m.st_gemm_f64(ta, tb, M, N, K, alpha, dA, A.shape[0], dB, B.shape[0], beta, C, M)
    m.st_sync()
    torch.cuda.synchronize()
    return _host(C, M)


def _op(X, t):
    return X.T if t else X


MODES = [0, 1]  # ST_DGEMM_SIMT, ST_DGEMM_OZAKI
TRANS = [(False, False), (True, False), (False, True), (True, True)]


# (M, N, K, bits): ragged against the 128 x 64 tiles and the K chunks (whole
# 64-wide stages, at most 448, chosen per product to fill the SMs); fewer
# rows or columns than one tile (TMA boxes past the last row); K shorter than
# one stage; K of the spatial dimension (128 chunks of 384)
SHAPES = [(200, 70, 600, 20), (5, 64, 49152, 15), (3000, 64, 20, 20), (130, 3, 20000, 15)]


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ta,tb", TRANS)
@pytest.mark.parametrize("shape", SHAPES)
def test_gemm_exact_on_integer_operands(mode, ta, tb, shape):
    rng = np.random.default_rng(7)
    M, N, K, bits = shape
    A = rng.integers(-2 ** bits, 2 ** bits, size=(M, K)).astype(np.float64)
    A *= np.ldexp(1.0, rng.integers(-30, 30, size=(M, 1)))  # per-row power-of-two scales
    A[min(3, M - 1)] = 0.0                                     # a zero row
    B = rng.integers(-2 ** bits, 2 ** bits, size=(K, N)).astype(np.float64)
    B[:, min(2, N - 1)] = 0.0                                  # a zero column
    # |terms| < 2^(2 bits) (times the row scale) and K 2^(2 bits) < 2^53: exact in FP64
    assert K * 2.0 ** (2 * bits) < 2.0 ** 53
    ref = A @ B
    m = _model(mode)
    got = _gemm(m, ta, tb, np.ascontiguousarray(_op(A, ta)), np.ascontiguousarray(_op(B, tb)))
    assert np.array_equal(got, ref)
    m.close()


@pytest.mark.parametrize("mode", MODES)
@pytest.mark.parametrize("ta,tb", TRANS)
def test_gemm_random_accuracy(mode, ta, tb):
    rng = np.random.default_rng(11)
    M, N, K = 300, 130, 1000
    A = rng.standard_normal((M, K)) * np.exp(rng.uniform(-20, 20, size=(M, 1)))
    B = rng.standard_normal((K, N)) * np.exp(rng.uniform(-20, 20, size=(1, N)))
    C0 = rng.standard_normal((M, N))
    alpha, beta = -1.5, 0.5
    ref = alpha * (A @ B) + beta * C0
    bound = abs(alpha) * (np.abs(A) @ np.abs(B)) + abs(beta) * np.abs(C0)
    m = _model(mode)
    got = _gemm(m, ta, tb, np.ascontiguousarray(_op(A, ta)), np.ascontiguousarray(_op(B, tb)), alpha, beta, C0)
    assert (np.abs(got - ref) <= 1e-14 * bound).all()
    m.close()


@pytest.mark.parametrize("shape", ["projection", "update"])
def test_gemm_pod_shapes_full_size(shape):
    # the two products of a block Gram-Schmidt pass at the 2-D S4 transport
    # size: L = W^T U (K = N = 49,152, split in 128 chunks of 384) and U -= W L
    rng = np.random.default_rng(3)
    N, r, b = 49152, 256, 64
    W = np.linalg.qr(rng.standard_normal((N, r)))[0]
    U = W @ rng.standard_normal((r, b)) + 1e-3 * rng.standard_normal((N, b))
    m0, m1 = _model(0), _model(1)
    if shape == "projection":
        ref = W.T @ U
        bound = np.abs(W.T) @ np.abs(U)
        outs = [_gemm(mm, True, False, W, U) for mm in (m0, m1)]
    else:
        L = W.T @ U
        ref = U - W @ L
        bound = np.abs(W) @ np.abs(L) + np.abs(U)
        outs = [_gemm(mm, False, False, W, L, -1.0, 1.0, U) for mm in (m0, m1)]
    for got in outs:
        assert (np.abs(got - ref) <= 1e-14 * bound).all()
    m0.close()
    m1.close()


def test_gemm_tensor_path_is_deterministic():
    rng = np.random.default_rng(5)
    A = rng.standard_normal((4000, 300))
    B = rng.standard_normal((4000, 90))
    m = _model(1)
    a = _gemm(m, True, False, A, B)
    b = _gemm(m, True, False, A, B)
    assert np.array_equal(a, b)
    m.close()


@pytest.mark.parametrize("mode", MODES)
def test_gemm_empty_and_k0(mode):
    torch = torch_mod()
    m = _model(mode)
    C0 = np.arange(12.0).reshape(4, 3)
    C = _dev(C0)
    m.st_gemm_f64(0, 0, 4, 3, 0, 1.0, None, 4, None, 1, 2.0, C, 4)  # K = 0: C = beta C
    m.st_sync()
    assert np.array_equal(_host(C, 4), 2.0 * C0)
    m.st_gemm_f64(0, 0, 0, 3, 5, 1.0, None, 1, None, 5, 0.0, C, 4)  # M = 0: nothing
    m.st_sync()
    torch.cuda.synchronize()
    m.close()


def test_gemm_tensor_path_reports_nonfinite_operands():
    import paper_1910_01260_gb300 as st
    rng = np.random.default_rng(9)
    A = rng.standard_normal((512, 256))
    A[17, 40] = np.nan
    B = rng.standard_normal((512, 128))
    m = _model(1)
    with pytest.raises(st.StError) as e:
        _gemm(m, True, False, A, B)
    assert e.value.code == st.ST_ERR_NONFINITE
    m.close()
