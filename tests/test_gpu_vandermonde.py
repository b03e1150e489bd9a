"""tr_vandermonde against the oracle's FP64 Horner product and closed forms.

Errors are normwise, against S[i][j] = sum_k |C[k][j]| |x_i|^k (the oracle
computes both Y and S):
  * TR_PREC_FP32 (Horner with fma): |y - y_ref| <= gamma_63 S (Higham,
    Sec. 5.1, u = 2^-24);
  * TR_PREC_BF16X3 (tensor cores): each power and coefficient is carried as
    two bf16 parts (about 2^-16 relative) and the dropped second-order terms
    are ~2^-16, so |y - y_ref| <= 1e-4 S is the pass bar (observed ~2e-5);
  * TR_PREC_BF16X6: three bf16 parts carry every FP32 value exactly and the
    dropped terms are ~2^-24; the bar is 1e-5 S (observed error printed).
Column results (sum / min / max of Y over the points) are checked against the
oracle's Y with bars scaled by sum_i S_ij (sums) and max_i S_ij (min / max),
and, at the full benchmark size, the column sums against the Faulhaber
closed form on a dyadic grid of points.  BF16 output equals the FP32 output
of the same path rounded to nearest even, bit for bit.  Identity-like and
binomial coefficient matrices pin the layout (a transposed operand or a wrong
core-matrix stride breaks them at once).  Row and column tails (m not a
multiple of 128, npoly not a multiple of 256) are covered.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import gamma

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

BAR = {0: 1e-4, 1: gamma(63) * 1.01, 2: 1e-5}  # by precision: x3, FP32, x6


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import binding, build
    build.build()
    binding.lib()
    return binding


def run(B, x, C, prec, out=torch.float32, cols=False):
    m, npoly = x.size, C.shape[1]
    y = torch.full((m, npoly), float("nan"), dtype=out, device="cuda") if out is not None else None
    ws = B.workspace(B.tr_vandermonde_workspace_size(m, npoly))
    ex = B.make_exec(ws)
    cs = [torch.full((npoly,), float("nan"), dtype=torch.float32, device="cuda") for _ in range(3)] if cols else [None] * 3
    xd = torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda()
    Cd = torch.from_numpy(np.ascontiguousarray(C, np.float32)).cuda()
    B.tr_vandermonde(xd, Cd, y, prec, ex, colsum=cs[0], colmin=cs[1], colmax=cs[2])
    B.tr_check(ex)
    if cols:
        return y, [c.cpu().numpy().astype(np.float64) for c in cs]
    return y


def normwise(orc, x, C, y, rows=None):
    ref, S = orc.vandermonde(x.astype(np.float64), C.astype(np.float64), rows=rows)
    got = y.cpu().float().numpy().astype(np.float64)
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
    assert e <= BAR[1], e


@pytest.mark.parametrize("prec", [0, 2], ids=["bf16x3", "bf16x6"])
@pytest.mark.parametrize("m,npoly,deg", [(128, 256, 31), (1280, 512, 31), (256, 256, 5), (1000, 300, 31),
                                         (33, 8, 31), (1, 4, 0)])
def test_split_normwise(orc, B, prec, m, npoly, deg):
    g = np.random.default_rng(7 * m + npoly)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, deg, npoly)
    y = run(B, x, C, prec)
    e, *_ = normwise(orc, x, C, y)
    print(f"precision {prec} {m}x{npoly}: max normwise error {e:.3g}")
    assert e <= BAR[prec], e


def test_large_points_and_low_degree(orc, B):
    """|x| around 20 with degree 8: powers above the degree are zero, so the
    product stays finite where the full 32 powers would overflow."""
    g = np.random.default_rng(12)
    x = g.uniform(18, 22, 256).astype(np.float32) * np.where(g.random(256) < 0.5, -1, 1).astype(np.float32)
    C = _coef(g, 8, 256)
    for prec in (0, 2):
        y = run(B, x, C, prec)
        e, *_ = normwise(orc, x, C, y)
        assert e <= BAR[prec], (prec, e)


@pytest.mark.parametrize("prec", [0, 2], ids=["bf16x3", "bf16x6"])
def test_bf16_output_is_rounded_fp32_output(B, prec):
    g = np.random.default_rng(5)
    m, npoly = 1000, 264
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, 31, npoly)
    y32 = run(B, x, C, prec)
    y16 = run(B, x, C, prec, out=torch.bfloat16)
    assert torch.equal(y16.view(torch.int16), y32.to(torch.bfloat16).view(torch.int16))


def _check_cols(orc, x, C, cols, bar):
    s, lo, hi = cols
    ref, S = orc.vandermonde(x.astype(np.float64), C.astype(np.float64))
    rs = np.array([math.fsum(ref[:, j]) for j in range(ref.shape[1])])
    scale_sum = S.sum(axis=0)
    scale_mm = S.max(axis=0)
    es = np.max(np.abs(s - rs) / scale_sum)
    emn = np.max(np.abs(lo - ref.min(axis=0)) / scale_mm)
    emx = np.max(np.abs(hi - ref.max(axis=0)) / scale_mm)
    return es, emn, emx


@pytest.mark.parametrize("prec", [0, 2], ids=["bf16x3", "bf16x6"])
@pytest.mark.parametrize("out", ["none", "f32", "bf16"])
@pytest.mark.parametrize("m,npoly", [(1000, 264), (128 * 41 + 5, 520), (7, 8)])
def test_column_results(orc, B, prec, out, m, npoly):
    g = np.random.default_rng(m + 3 * npoly + prec)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, 31, npoly)
    dt = {"none": None, "f32": torch.float32, "bf16": torch.bfloat16}[out]
    y, cols = run(B, x, C, prec, out=dt, cols=True)
    es, emn, emx = _check_cols(orc, x, C, cols, BAR[prec])
    print(f"precision {prec}, out {out}, {m}x{npoly}: column sum {es:.3g}, min {emn:.3g}, max {emx:.3g}")
    assert es <= BAR[prec] and emn <= BAR[prec] and emx <= BAR[prec], (es, emn, emx)
    if out == "f32":
        # the column results are those of the written Y (same FP32 tile values)
        yy = y.cpu().numpy().astype(np.float64)
        assert np.array_equal(cols[1], yy.min(axis=0)) and np.array_equal(cols[2], yy.max(axis=0))
    _, again = run(B, x, C, prec, out=dt, cols=True)
    assert all(np.array_equal(a, b) for a, b in zip(cols, again))  # deterministic


def test_column_results_any_npoly_without_output(orc, B):
    g = np.random.default_rng(21)
    m, npoly = 640, 257
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, 31, npoly)
    _, cols = run(B, x, C, 0, out=None, cols=True)
    es, emn, emx = _check_cols(orc, x, C, cols, BAR[0])
    assert es <= BAR[0] and emn <= BAR[0] and emx <= BAR[0], (es, emn, emx)


def test_identity_and_binomial(orc, B):
    """Column j < 32 of an identity-like C is x^j; column 32 holds binomial
    coefficients, so it is (1 + x)^31.  Remaining columns random."""
    m, npoly, deg = 256, 256, 31
    g = np.random.default_rng(3)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, deg, npoly)
    C[:, :32] = np.eye(32)
    C[:, 32] = [math.comb(31, k) for k in range(32)]
    xd = x.astype(np.float64)
    for prec in (0, 2):
        y = run(B, x, C, prec).cpu().numpy().astype(np.float64)
        for j in range(32):
            assert np.all(np.abs(y[:, j] - xd ** j) <= BAR[prec] * np.abs(xd) ** j + 1e-38)
        S = (1 + np.abs(xd)) ** 31
        assert np.all(np.abs(y[:, 32] - (1 + xd) ** 31) <= BAR[prec] * S)


def test_persistent_tiles_and_column_reload(orc, B):
    """More tiles than CTAs and several column tiles per CTA range, with and
    without output (without Y the transposed product walks 128-polynomial
    blocks, several per CTA range as well)."""
    m, npoly = 128 * 700, 768
    g = np.random.default_rng(11)
    x = g.uniform(-1, 1, m).astype(np.float32)
    C = _coef(g, 31, npoly)
    y, cols = run(B, x, C, 0, cols=True)
    rows = np.arange(0, m, 37)
    e, *_ = normwise(orc, x, C, y, rows=rows)
    assert e <= BAR[0], e
    yy = y.cpu().numpy().astype(np.float64)
    assert np.array_equal(cols[1], yy.min(axis=0)) and np.array_equal(cols[2], yy.max(axis=0))
    s_from_y = np.array([math.fsum(yy[:, j]) for j in range(npoly)])
    assert np.all(np.abs(cols[0] - s_from_y) <= 1e-6 * np.abs(yy).sum(axis=0))
    for prec in (0, 2):
        _, alone = run(B, x, C, prec, out=None, cols=True)
        es, emn, emx = _check_cols(orc, x, C, alone, BAR[prec])
        print(f"precision {prec}, column results alone, {m}x{npoly}: sum {es:.3g}, min {emn:.3g}, max {emx:.3g}")
        assert es <= BAR[prec] and emn <= BAR[prec] and emx <= BAR[prec], (es, emn, emx)


def _dyadic_power_sums(N, deg):
    """P_k = sum_i x_i^k over x_i = (2i + 1 - N) / N, exactly (Faulhaber)."""
    from tests.test_oracle_pins import _dyadic_poly_sum
    return [_dyadic_poly_sum([0] * k + [1], N) for k in range(deg + 1)]


def test_full_size_sampled_rows(orc, B):
    """The benchmark size, 2^20 points x 4096 polynomials of degree 31, checked
    on every 2048th row against the oracle (FP32 Horner and both splits)."""
    x, C = I.vandermonde()
    rows = np.arange(0, x.size, 2048)
    for prec in (B.TR_PREC_BF16X3, B.TR_PREC_BF16X6, B.TR_PREC_FP32):
        y = run(B, x, C, prec)
        e, *_ = normwise(orc, x, C, y, rows=rows)
        print(f"precision {prec}: max normwise error {e:.3g}")
        assert e <= BAR[prec], e
        del y
        torch.cuda.empty_cache()


def test_full_size_column_sums_closed_form(B):
    """At the benchmark size (2^20 points, 4096 polynomials of degree 31, the
    benchmark's coefficients) on the dyadic grid x_i = (2i + 1 - N) / N: the
    fused column sums against sum_k C_kj P_k with the power sums P_k in closed
    form, normwise against sum_k |C_kj| sum_i |x_i|^k."""
    N = 1 << 20
    _, C = I.vandermonde()
    x = ((2.0 * np.arange(N) + 1 - N) / N).astype(np.float32)
    P = _dyadic_power_sums(N, 31)
    # sum_i |x_i|^k: the grid is symmetric, so for odd k it is twice the sum over the positive half
    half = ((2.0 * np.arange(N // 2, N) + 1 - N) / N)
    abs_odd = {k: 2 * math.fsum(half ** k) for k in range(1, 32, 2)}
    Pabs = [float(P[k]) if k % 2 == 0 else abs_odd[k] for k in range(32)]
    Cf = [[Fraction(float(c)) for c in row] for row in C.astype(np.float64)]
    exact = np.array([float(sum(Cf[k][j] * P[k] for k in range(32))) for j in range(C.shape[1])])
    scale = np.abs(C.astype(np.float64)).T @ np.array(Pabs)
    for prec in (B.TR_PREC_BF16X3, B.TR_PREC_BF16X6):
        _, cols = run(B, x, C, prec, out=None, cols=True)
        e = np.max(np.abs(cols[0] - exact) / scale)
        print(f"precision {prec}: full-size column sums, max normwise error {e:.3g}")
        assert e <= BAR[prec], e


def test_validation(B):
    x = np.zeros(100, np.float32)
    with pytest.raises(B.TrError) as e:
        run(B, x, np.zeros((32, 258), np.float32), B.TR_PREC_BF16X3)  # FP32 output needs npoly % 4 == 0
    assert e.value.status == 2
    with pytest.raises(B.TrError) as e:
        run(B, x, np.zeros((32, 260), np.float32), B.TR_PREC_BF16X3, out=torch.bfloat16)  # BF16: npoly % 8 == 0
    assert e.value.status == 2
    with pytest.raises(B.TrError) as e:
        run(B, x, np.zeros((32, 256), np.float32), B.TR_PREC_BF16X3, out=None)  # nothing requested
    assert e.value.status == 1
    with pytest.raises(B.TrError) as e:
        run(B, x, np.zeros((32, 256), np.float32), B.TR_PREC_FP32, out=torch.bfloat16)
    assert e.value.status == 3
