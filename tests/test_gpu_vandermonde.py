"""tr_vandermonde against the oracle's FP64 Horner product.

Errors are normwise, against S[i][j] = sum_k |C[k][j]| |x_i|^k (the oracle
computes both Y and S):
  * TR_PREC_FP32 (Horner with fma): |y - y_ref| <= gamma_63 S (Higham,
    Sec. 5.1, u = 2^-24);
  * TR_PREC_BF16X3 (tensor cores): each power and coefficient is carried as a
    bf16 pair to about 2^-17 relative and the dropped Vl*Cl term is ~2^-18,
    so |y - y_ref| <= 1e-4 S is the pass bar and the observed maximum is
    printed (expected ~1e-5).
Identity-like and binomial coefficient matrices pin the layout (a transposed
operand or a wrong core-matrix stride breaks them at once).
"""
import math

import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import gamma

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import binding, build
    build.build()
    binding.lib()
    return binding


def run(B, x, C, prec):
    m, npoly = x.size, C.shape[1]
    y = torch.full((m, npoly), float("nan"), dtype=torch.float32, device="cuda")
    ws = B.workspace(256)
    ex = B.make_exec(ws)
    B.tr_vandermonde(torch.from_numpy(x).cuda(), torch.from_numpy(np.ascontiguousarray(C, np.float32)).cuda(), y,
                     prec, ex)
    B.tr_check(ex)
    return y


def normwise(orc, x, C, y, rows=None):
    ref, S = orc.vandermonde(x.astype(np.float64), C.astype(np.float64), rows=rows)
    got = y.cpu().numpy().astype(np.float64)
    if rows is not None:
        got = got[rows]
    assert np.all(np.isfinite(got))
    return np.max(np.abs(got - ref) / np.maximum(S, 1e-300)), got, ref, S


def _coef(g, deg, npoly):
    return I.f32_exact(g.standard_normal((deg + 1, npoly)) / (np.arange(deg + 1)[:, None] + 1.0))


@pytest.mark.parametrize("m,npoly,deg", [(1000, 300, 31), (33, 7, 31), (4096, 256, 8), (1, 1, 0)])
def test_fp32_within_horner_bound(orc, B, m, npoly, deg):
    g = np.random.default_rng(m + npoly)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, deg, npoly)
    y = run(B, x, C, B.TR_PREC_FP32)
    e, *_ = normwise(orc, x, C, y)
    assert e <= gamma(63) * 1.01, e


@pytest.mark.parametrize("m,npoly,deg", [(128, 256, 31), (1280, 512, 31), (256, 256, 5)])
def test_bf16x3_normwise(orc, B, m, npoly, deg):
    g = np.random.default_rng(7 * m + npoly)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, deg, npoly)
    y = run(B, x, C, B.TR_PREC_BF16X3)
    e, *_ = normwise(orc, x, C, y)
    print(f"bf16x3 max normwise error {e:.3g}")
    assert e <= 1e-4, e


def test_bf16x3_identity_and_binomial(orc, B):
    """Column j < 32 of an identity-like C is x^j; column 32 holds binomial
    coefficients, so it is (1 + x)^31.  Remaining columns random."""
    m, npoly, deg = 256, 256, 31
    g = np.random.default_rng(3)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, deg, npoly)
    C[:, :32] = np.eye(32)
    C[:, 32] = [math.comb(31, k) for k in range(32)]
    y = run(B, x, C, B.TR_PREC_BF16X3).cpu().numpy().astype(np.float64)
    xd = x.astype(np.float64)
    for j in range(32):
        assert np.all(np.abs(y[:, j] - xd ** j) <= 1e-4 * np.abs(xd) ** j + 1e-38)
    S = (1 + np.abs(xd)) ** 31
    assert np.all(np.abs(y[:, 32] - (1 + xd) ** 31) <= 1e-4 * S)


def test_bf16x3_persistent_tiles_and_column_reload(orc, B):
    """More tiles than CTAs and several column tiles per CTA range."""
    m, npoly = 128 * 700, 768
    g = np.random.default_rng(11)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, 31, npoly)
    y = run(B, x, C, B.TR_PREC_BF16X3)
    rows = np.arange(0, m, 37)
    e, *_ = normwise(orc, x, C, y, rows=rows)
    assert e <= 1e-4, e


def test_full_size_sampled_rows(orc, B):
    """The benchmark size, 2^20 points x 4096 polynomials of degree 31, checked
    on every 2048th row against the oracle (both precisions)."""
    x, C = I.vandermonde()
    rows = np.arange(0, x.size, 2048)
    for prec, bar in ((B.TR_PREC_BF16X3, 1e-4), (B.TR_PREC_FP32, gamma(63) * 1.01)):
        y = run(B, x, C, prec)
        e, *_ = normwise(orc, x, C, y, rows=rows)
        print(f"precision {prec}: max normwise error {e:.3g}")
        assert e <= bar, e
        del y
        torch.cuda.empty_cache()


def test_validation(B):
    x = np.zeros(100, np.float32)
    C = np.zeros((32, 256), np.float32)
    with pytest.raises(B.TrError) as e:
        run(B, x, C, B.TR_PREC_BF16X3)  # m not a multiple of 128
    assert e.value.status == 3
