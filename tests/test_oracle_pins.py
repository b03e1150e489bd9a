"""Pins of the CPU oracle against things other than itself (CPU only).

Each oracle function is checked against at least one of: a library routine
with a correct-rounding guarantee (math.fsum, numpy.float32 of an exact
integer, numpy.cbrt), a closed form (Faulhaber power sums, telescoping series,
full-domain bijection sums), an independent formulation (xorshift as a GF(2)
matrix, splitmix inverted with constants derived from sqrt/golden-ratio by
integer square roots), or a brute force with Python Fractions on tiny inputs.
The cases are chosen so that a dropped term, a wrong sign or index, or a
transposed operand fails at least one of them.
"""
import math
from fractions import Fraction

import numpy as np
import pytest

U64 = 1 << 64
M32 = (1 << 32) - 1


# --------------------------------------------------------------------------
# exact summation
# --------------------------------------------------------------------------

def _wide_doubles(seed, n):
    g = np.random.default_rng(seed)
    v = g.standard_normal(n) * np.exp2(g.integers(-80, 80, n))
    v[::7] *= -1e-300  # tiny values, some subnormal after scaling
    v[3::11] = np.exp2(g.integers(-1074, -1022, v[3::11].size)).astype(np.float64)
    return v


@pytest.mark.parametrize("seed", range(6))
def test_exact_sum_matches_fsum(orc, seed):
    """math.fsum is correctly rounded (Shewchuk); the oracle must agree bit for bit."""
    v = _wide_doubles(seed, 2000)
    assert orc.exact_sum(v) == math.fsum(v)
    # heavy cancellation
    w = np.concatenate([v, -v[::-1], [1e-300, 3.0]])
    assert orc.exact_sum(w) == math.fsum(w) == 3.0 + 1e-300
    # order independence
    p = np.random.default_rng(seed + 100).permutation(v)
    assert orc.exact_sum(p) == orc.exact_sum(v)


def test_exact_sum_edge_cases(orc):
    assert orc.exact_sum([]) == 0.0
    assert orc.exact_sum([5e-324]) == 5e-324
    assert orc.exact_sum([5e-324, 5e-324]) == 1e-323
    assert orc.exact_sum([1.7976931348623157e308, -1.7976931348623157e308, 1.0]) == 1.0
    # ties to even at double precision: 1 + 2^-53 -> 1, 1 + 3*2^-53 -> 1 + 2^-51
    assert orc.exact_sum([1.0, 2.0 ** -53]) == 1.0
    assert orc.exact_sum([1.0, 2.0 ** -53, 2.0 ** -52]) == 1.0 + 2.0 ** -51
    assert orc.exact_sum([1.0, 2.0 ** -53, 2.0 ** -105]) == 1.0 + 2.0 ** -52  # sticky bit


def test_exact_sum_float_rounding(orc):
    """p = 24: for sums exactly representable in double, rounding the double to
    float32 is a single correct rounding, so numpy's cast is the reference."""
    g = np.random.default_rng(7)
    for _ in range(200):
        k = g.integers(1, 40)
        v = g.integers(-(1 << 30), 1 << 30, k).astype(np.float64) * 2.0 ** int(g.integers(-30, 10))
        s = math.fsum(v)
        assert Fraction(s) == sum(Fraction(x) for x in v)  # exact in double
        assert orc.exact_sum(v, 24) == float(np.float32(s))
    # explicit float ties: 1 + 2^-24 -> 1 ; 1 + 3*2^-24 -> 1 + 2^-22
    assert orc.exact_sum([1.0, 2.0 ** -24], 24) == 1.0
    assert orc.exact_sum([1.0, 2.0 ** -24, 2.0 ** -23], 24) == 1.0 + 2.0 ** -22
    assert orc.exact_sum([1.0, 2.0 ** -24, 2.0 ** -80], 24) == 1.0 + 2.0 ** -23
    # float subnormal quantum 2^-149
    assert orc.exact_sum([2.0 ** -150, 2.0 ** -151], 24) == 2.0 ** -149
    assert orc.exact_sum([2.0 ** -150], 24) == 0.0  # tie to even (0)


# --------------------------------------------------------------------------
# Horner
# --------------------------------------------------------------------------

def _faulhaber(p, n):
    """sum_{i=0}^{n-1} i^p by Faulhaber's formula (Bernoulli numbers, B1 = -1/2)."""
    B = [Fraction(1)]
    for m in range(1, p + 1):
        B.append(-sum(math.comb(m + 1, j) * B[j] for j in range(m)) / (m + 1))
    return sum(math.comb(p + 1, j) * B[j] * Fraction(n) ** (p + 1 - j) for j in range(p + 1)) / (p + 1)


def _dyadic_poly_sum(coef, N):
    """Exact sum over x_i = (2i+1-N)/N, i < N, of sum_k c_k x^k, via power sums."""
    total = Fraction(0)
    for k, c in enumerate(coef):
        # (2i + 1 - N)^k expanded by the binomial theorem, then Faulhaber in i
        s = Fraction(0)
        for j in range(k + 1):
            s += math.comb(k, j) * Fraction(2) ** j * Fraction(1 - N) ** (k - j) * _faulhaber(j, N)
        total += Fraction(c) * s / Fraction(N) ** k
    return total


@pytest.mark.parametrize("coef", [[3, -2, 5], [1, 0, -7, 2], [-4, 9, 1, -3, 2], [0, 0, 0, 1, 0]])
def test_horner_dyadic_closed_form(orc, coef):
    """On the dyadic grid with small integer coefficients every Horner step is
    exact in FP64, so the oracle's reduction must equal the Faulhaber closed
    form rounded once -- bit for bit."""
    N = 1 << 10
    x = (2.0 * np.arange(N) + 1 - N) / N
    m = orc.MapSpec("horner", coef)
    s, lo, hi = orc.reduce_float(m, x)
    assert s == float(_dyadic_poly_sum(coef, N))
    vals = [sum(Fraction(c) * Fraction(xi) ** k for k, c in enumerate(coef)) for xi in x[::97]]
    assert np.array_equal(orc.map_values(m, x[::97]), np.array([float(v) for v in vals]))
    exact = [sum(Fraction(c) * Fraction(xi) ** k for k, c in enumerate(coef)) for xi in x]
    assert lo == float(min(exact)) and hi == float(max(exact))


def test_horner_error_bound(orc):
    """Random degree-31 polynomials: |p_hat - p| <= gamma_{2d} sum |c_k||x|^k
    (Higham, Accuracy and Stability, Sec. 5.1), with p exact by Fractions."""
    g = np.random.default_rng(3)
    d = 31
    c = g.standard_normal(d + 1)
    x = g.uniform(-1.2, 1.2, 64)
    y = orc.map_values(orc.MapSpec("horner", c), x)
    u = 2.0 ** -53
    gam = 2 * d * u / (1 - 2 * d * u)
    for xi, yi in zip(x, y):
        exact = sum(Fraction(ck) * Fraction(xi) ** k for k, ck in enumerate(c))
        scale = sum(abs(ck) * abs(xi) ** k for k, ck in enumerate(c))
        assert abs(Fraction(yi) - exact) <= Fraction(gam * scale)


def test_horner_fma_sequence_bruteforce(orc):
    """Tiny inputs: every step rounds once (fma), simulated with Fractions."""
    g = np.random.default_rng(5)
    c = g.standard_normal(9)
    x = g.uniform(-1, 1, 16)
    y = orc.map_values(orc.MapSpec("horner", c), x)
    for xi, yi in zip(x, y):
        p = Fraction(c[-1])
        for ck in c[-2::-1]:
            p = Fraction(float(p * Fraction(xi) + Fraction(ck)))  # float(Fraction) rounds correctly
        assert float(p) == yi


# --------------------------------------------------------------------------
# rational, square, Newton
# --------------------------------------------------------------------------

def test_rational_telescoping(orc):
    """P = 1, Q = x^2 + x at x = 1..n:  f(i) = 1/i - 1/(i+1), the sum telescopes
    to 1 - 1/(n+1); each FP64 term is off by <= u f(i), so the total is within 2u."""
    n = 5000
    x = np.arange(1, n + 1, dtype=np.float64)
    m = orc.MapSpec("rational", [1.0], [0.0, 1.0, 1.0])
    s, lo, hi = orc.reduce_float(m, x)
    assert abs(s - (1 - 1 / (n + 1))) <= 2 * 2.0 ** -53
    assert hi == 0.5 and lo == 1.0 / (n * (n + 1.0))
    # prefix-wise, rounded to float: 1 - 1/(k+1) within one float ulp
    y = orc.scan_float(m, x, 24)
    ref = 1 - 1 / (np.arange(1, n + 1) + 1.0)
    assert np.all(np.abs(y - ref) <= np.spacing(np.float32(ref)).astype(np.float64))
    # operands not swapped: Q/P would give i^2 + i
    assert orc.map_values(m, [3.0])[0] == 1.0 / 12.0


def test_rational_error_bound(orc):
    g = np.random.default_rng(9)
    cp = g.standard_normal(7)
    cq = np.array([1.0, 0, 0.7, 0, 0.3, 0, 0.2])
    x = g.standard_normal(64)
    y = orc.map_values(orc.MapSpec("rational", cp, cq), x)
    for xi, yi in zip(x, y):
        P = sum(Fraction(c) * Fraction(xi) ** k for k, c in enumerate(cp))
        Q = sum(Fraction(c) * Fraction(xi) ** k for k, c in enumerate(cq))
        sp = sum(abs(c) * abs(xi) ** k for k, c in enumerate(cp))
        # Q >= 1 and its Horner error is tiny: bound (gamma_12 sp + |P| gamma_13)/Q
        bound = (13 * 2.0 ** -53) * (sp + abs(float(P / Q)) * sum(abs(c) * abs(xi) ** k for k, c in enumerate(cq))) \
            / float(Q) + 2.0 ** -53 * abs(float(P / Q))
        assert abs(Fraction(yi) - P / Q) <= Fraction(bound * 1.01)


def test_square_prefix_closed_form(orc):
    """x_i = i: prefix of i^2 is k(k+1)(2k+1)/6 (exact integers), rounded once."""
    n = 4096
    x = np.arange(1, n + 1, dtype=np.float64)
    m = orc.MapSpec("square")
    y53 = orc.scan_float(m, x, 53)
    k = np.arange(1, n + 1, dtype=np.int64)
    ref = k * (k + 1) * (2 * k + 1) // 6
    assert np.array_equal(y53, ref.astype(np.float64))
    y24 = orc.scan_float(m, x, 24)
    assert np.array_equal(y24, ref.astype(np.float64).astype(np.float32).astype(np.float64))
    assert orc.reduce_float(m, x)[0] == float(ref[-1])


def test_newton_cbrt(orc):
    m = orc.MapSpec("newton_cbrt", iters=6)
    # converged region: equals the library cube root within 2 ulps
    x = np.linspace(0.5, 2.0, 1001)
    y = orc.map_values(m, np.concatenate([x, -x]))
    ref = np.cbrt(np.concatenate([x, -x]))
    assert np.all(np.abs(y - ref) <= 2 * np.spacing(np.abs(ref)))
    # odd symmetry holds exactly
    assert np.array_equal(y[:1001], -y[1001:])
    # x = 0: y_k = (2/3)^k, the iterate, not cbrt(0)
    assert abs(orc.map_values(m, [0.0])[0] - (2.0 / 3.0) ** 6) <= 1e-15
    # far from 1 the iterate has not converged; brute force with per-op rounding
    for xi in [1000.0, -1e-3, 37.5, 1e6]:
        yy = Fraction(math.copysign(1.0, xi))
        for _ in range(6):
            yy2 = Fraction(float(yy * yy))
            q = Fraction(float(Fraction(xi) / yy2))
            t = Fraction(float(2 * yy + q))
            yy = Fraction(float(t / 3))
        assert orc.map_values(m, [xi])[0] == float(yy)
    assert orc.map_values(orc.MapSpec("newton_cbrt", iters=40), [1e6])[0] == pytest.approx(100.0, rel=1e-15)


# --------------------------------------------------------------------------
# integer mixers
# --------------------------------------------------------------------------

def _gf2_shift_matrix(shift):
    """32x32 matrix over GF(2) of x -> x << s (s > 0) or x >> -s (s < 0); bit 0 = lsb."""
    M = np.zeros((32, 32), dtype=np.uint8)
    for j in range(32):
        i = j + shift
        if 0 <= i < 32:
            M[i, j] = 1
    return M


def test_xorshift32_gf2_matrix(orc):
    """xorshift32 is the linear map (I + L^5)(I + R^17)(I + L^13) over GF(2)."""
    I = np.eye(32, dtype=np.uint8)
    T = ((I + _gf2_shift_matrix(5)) @ (I + _gf2_shift_matrix(-17)) @ (I + _gf2_shift_matrix(13))) % 2
    g = np.random.default_rng(11)
    x = g.integers(0, 1 << 32, 4000, dtype=np.uint64).astype(np.uint32)
    bits = ((x[:, None] >> np.arange(32, dtype=np.uint32)) & 1).astype(np.int64)
    ybits = (bits @ T.T.astype(np.int64)) % 2
    ref = (ybits.astype(np.uint64) << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)
    y = orc.map_values(orc.MapSpec("xorshift32"), x)
    assert np.array_equal(y, ref)
    assert orc.map_values(orc.MapSpec("xorshift32"), np.array([0], np.uint32))[0] == 0


def _splitmix_constants():
    """Weyl increment floor(2^32/phi) = floor(2^31 sqrt 5) - 2^31; multipliers
    floor(frac(sqrt 2) 2^32) and floor(frac(sqrt 3) 2^32), by integer sqrt."""
    inc = math.isqrt(5 << 62) - (1 << 31)
    m1 = math.isqrt(2 << 64) - (1 << 32)
    m2 = math.isqrt(3 << 64) - (1 << 32)
    return inc, m1, m2


def _splitmix_inverse(y):
    inc, m1, m2 = _splitmix_constants()
    z = y ^ (y >> 16)                      # x ^= x>>16 is an involution on 32 bits
    z = (z * pow(m2, -1, 1 << 32)) & M32
    z = z ^ (z >> 13) ^ (z >> 26)          # inverse of x ^= x>>13
    z = (z * pow(m1, -1, 1 << 32)) & M32
    z = z ^ (z >> 16)
    return (z - inc) & M32


def test_splitmix32_inverse(orc):
    inc, m1, m2 = _splitmix_constants()
    assert m1 % 2 == 1 and m2 % 2 == 1
    g = np.random.default_rng(12)
    x = g.integers(0, 1 << 32, 3000, dtype=np.uint64).astype(np.uint32)
    x[:4] = [0, 1, M32, 1 << 31]
    y = orc.map_values(orc.MapSpec("splitmix32"), x)
    for xi, yi in zip(x.tolist(), y.tolist()):
        assert _splitmix_inverse(yi) == xi


@pytest.mark.slow
@pytest.mark.parametrize("kind", ["xorshift32", "splitmix32"])
def test_mixer_full_domain_sum(orc, kind):
    """Both mixers are bijections of the 32-bit integers, so over the whole
    domain the sum of f(x) is sum x = 2^31 (2^32 - 1)."""
    assert orc.mixer_range_sum(kind, 0, 1 << 32) == (1 << 31) * ((1 << 32) - 1)


# --------------------------------------------------------------------------
# u32 reductions and scans
# --------------------------------------------------------------------------

@pytest.mark.parametrize("kind", ["xorshift32", "splitmix32", "identity"])
def test_u32_reduce_and_scans(orc, kind):
    g = np.random.default_rng(13)
    x = g.integers(0, 1 << 32, 5001, dtype=np.uint64).astype(np.uint32)
    m = orc.MapSpec(kind)
    f = orc.map_values(m, x)
    s, lo, hi = orc.reduce_u32(m, x)
    assert s == sum(int(v) for v in f)
    assert lo == int(f.min()) and hi == int(f.max())
    y32 = orc.scan_u32(m, x)
    assert np.array_equal(y32, np.cumsum(f, dtype=np.uint32))
    y64 = orc.scan_u32_u64(m, x)
    assert np.array_equal(y64, np.cumsum(f.astype(np.uint64)))
    assert int(y64[-1]) == s and int(y32[-1]) == s % (1 << 32)
    assert orc.reduce_u32(m, x[:0]) == (0, M32, 0)


# --------------------------------------------------------------------------
# segmented reduction
# --------------------------------------------------------------------------

def test_segmented_reduce(orc):
    g = np.random.default_rng(14)
    x = g.standard_normal(3000).astype(np.float32)
    m = orc.MapSpec("rational", g.standard_normal(7), [1.0, 0, 0.5, 0, 0.25, 0, 0.125])
    off = np.array([0, 0, 1, 1, 500, 501, 1999, 3000, 3000], dtype=np.int64)
    sums, mins, maxs = orc.segmented_reduce_float(m, x, off)
    f = orc.map_values(m, x)
    for s in range(off.size - 1):
        seg = f[off[s]:off[s + 1]]
        assert sums[s] == math.fsum(seg)
        if seg.size:
            assert mins[s] == seg.min() and maxs[s] == seg.max()
        else:
            assert mins[s] == np.inf and maxs[s] == -np.inf and sums[s] == 0.0
    full = orc.reduce_float(m, x)
    one = orc.segmented_reduce_float(m, x, np.array([0, 3000]))
    assert one[0][0] == full[0] and one[1][0] == full[1] and one[2][0] == full[2]


# --------------------------------------------------------------------------
# Vandermonde
# --------------------------------------------------------------------------

def test_vandermonde_identity_and_binomial(orc):
    g = np.random.default_rng(15)
    x = g.uniform(-1, 1, 40)
    deg = 31
    # C = identity-like: column j is the monomial x^j
    C = np.zeros((deg + 1, deg + 1))
    np.fill_diagonal(C, 1.0)
    Y, S = orc.vandermonde(x, C)
    for j in range(deg + 1):
        ref = np.array([float(Fraction(xi) ** j) for xi in x])
        assert np.all(np.abs(Y[:, j] - ref) <= (j + 1) * 2.0 ** -53 * np.abs(ref))
    # binomial coefficients: column is (1 + x)^31
    Cb = np.array([[math.comb(deg, k)] for k in range(deg + 1)], dtype=np.float64)
    Yb, Sb = orc.vandermonde(x, Cb)
    ref = np.array([float((1 + Fraction(xi)) ** deg) for xi in x])
    assert np.all(np.abs(Yb[:, 0] - ref) <= 2 * deg * 2.0 ** -53 * Sb[:, 0] * 1.01)
    assert np.allclose(Sb[:, 0], (1 + np.abs(x)) ** deg, rtol=1e-13)
    # row subset selects rows
    Ys = orc.vandermonde(x, C, rows=[3, 7], with_scale=False)
    assert np.array_equal(Ys, Y[[3, 7]])


def test_vandermonde_dyadic_column_sums(orc):
    """Column sums over the dyadic grid equal the Faulhaber closed form (exact
    Horner steps with small integer coefficients)."""
    N = 1 << 8
    x = (2.0 * np.arange(N) + 1 - N) / N
    C = np.array([[1, 2], [-3, 0], [2, 5], [0, -1]], dtype=np.float64)  # deg 3, 2 polys
    Y = orc.vandermonde(x, C, with_scale=False)
    for j in range(2):
        assert math.fsum(Y[:, j]) == float(_dyadic_poly_sum(C[:, j].tolist(), N))


def test_scan_sampled_matches_full_scan(orc):
    """The sampled prefix routine returns exactly the full scan's values."""
    g = np.random.default_rng(16)
    x = g.uniform(0, 1, 20000).astype(np.float32)
    m = orc.MapSpec("square")
    full = orc.scan_float(m, x, 24)
    pos = np.sort(g.choice(x.size, 300, replace=False))
    assert np.array_equal(orc.scan_float_sampled(m, x, pos, 24), full[pos])


# --------------------------------------------------------------------------
# multi-threaded drivers and binary16 widening
# --------------------------------------------------------------------------

def test_widen_f16_all_patterns(orc):
    """Every binary16 bit pattern widens to numpy's exact float16 -> float64 value."""
    bits = np.arange(1 << 16, dtype=np.uint16)
    ref = bits.view(np.float16).astype(np.float64)
    got = orc.widen_f16(bits)
    nan = np.isnan(ref)
    assert np.array_equal(np.isnan(got), nan)
    assert np.array_equal(got[~nan].view(np.int64), ref[~nan].view(np.int64))


@pytest.mark.parametrize("threads", [1, 2, 3, 8])
def test_reduce_mt_equals_single_thread(orc, threads):
    """The threaded full reduction merges exact accumulators: the same bits as
    the single-thread oracle for any thread count, any storage type; its sum
    of |f| equals math.fsum of |f|."""
    g = np.random.default_rng(threads)
    m = orc.MapSpec("rational", g.standard_normal(7), [1.0, 0.0, 0.7, 0.0, 0.2, 0.0, 0.05])
    for dt in (np.float64, np.float32, np.float16):
        x = g.standard_normal(100_003).astype(dt)
        s, lo, hi, sa = orc.reduce_float_mt(m, x, threads)
        assert (s, lo, hi) == orc.reduce_float(m, x.astype(np.float64))
        assert sa == math.fsum(np.abs(orc.map_values(m, x.astype(np.float64))))
    assert orc.reduce_float_mt(m, np.zeros(0), threads) == (0.0, np.inf, -np.inf, 0.0)


@pytest.mark.parametrize("threads", [1, 2, 5, 8])
def test_segreduce_mt_equals_single_thread(orc, threads):
    """Threads take whole segments: the same bits as the single-thread
    segmented oracle (empty segments included), and the per-segment sum of
    |f| equals math.fsum of |f| over the segment."""
    g = np.random.default_rng(10 + threads)
    n = 50_000
    x = g.uniform(-2, 2, n).astype(np.float32)
    cut = np.sort(g.integers(0, n, 300))
    off = np.concatenate([[0, 0], cut, [n, n]]).astype(np.int64)
    m = orc.MapSpec("horner", g.standard_normal(9))
    x64 = x.astype(np.float64)
    sums, mins, maxs, abss = orc.segmented_reduce_float_mt(m, x, off, threads)
    rs, rlo, rhi = orc.segmented_reduce_float(m, x64, off)
    assert np.array_equal(sums, rs) and np.array_equal(mins, rlo) and np.array_equal(maxs, rhi)
    f = np.abs(orc.map_values(m, x64))
    ref_abs = [math.fsum(f[a:b]) for a, b in zip(off[:-1], off[1:])]
    assert np.array_equal(abss, np.array(ref_abs))


def test_exclusive_scans(orc):
    """Exclusive scans: y_0 = 0 and y_i equals the inclusive scan at i - 1 (the
    same exact prefix), and for f = x^2 on x = 0..n-1 the closed form
    sum_{j<i} j^2 = (i-1) i (2i-1) / 6."""
    g = np.random.default_rng(3)
    x = g.integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    for kind in ("xorshift32", "splitmix32"):
        m = orc.MapSpec(kind)
        for fn in (orc.scan_u32, orc.scan_u32_u64):
            inc, exc = fn(m, x), fn(m, x, exclusive=True)
            assert exc[0] == 0 and np.array_equal(exc[1:], inc[:-1])
    n = 3000
    i = np.arange(n, dtype=np.float64)
    exc = orc.scan_float(orc.MapSpec("square"), i, 53, exclusive=True)
    closed = np.array([(k - 1) * k * (2 * k - 1) // 6 for k in range(n)], dtype=np.float64)
    assert np.array_equal(exc, closed)
    xf = g.standard_normal(4000)
    m = orc.MapSpec("rational", [1.0, -2.0, 0.5], [1.0, 0.0, 0.3])
    inc, exc = orc.scan_float(m, xf, 24), orc.scan_float(m, xf, 24, exclusive=True)
    assert exc[0] == 0.0 and np.array_equal(exc[1:], inc[:-1])


# --------------------------------------------------------------------------
# binary32 evaluation of the maps
# --------------------------------------------------------------------------

def _rn32(fr: Fraction) -> float:
    """Round a rational to the nearest binary32 value, ties to even (subnormals included)."""
    if fr == 0:
        return 0.0
    sign = -1.0 if fr < 0 else 1.0
    a = abs(fr)
    e = a.numerator.bit_length() - a.denominator.bit_length()
    if Fraction(2) ** e > a:
        e -= 1
    q = max(e - 23, -149)
    m = a / Fraction(2) ** q
    n = m.numerator // m.denominator
    r = m - n
    if r > Fraction(1, 2) or (r == Fraction(1, 2) and n % 2 == 1):
        n += 1
    return sign * float(n) * 2.0 ** q


def _f32_values(g, k, scale=1.0):
    return (g.standard_normal(k) * scale).astype(np.float32).astype(np.float64)


def test_map_f32_bruteforce(orc):
    """Every binary32 map equals its operation sequence carried out with exact
    rationals and one round-to-nearest-even to binary32 per operation."""
    g = np.random.default_rng(32)
    x = np.concatenate([_f32_values(g, 60, 2.0), [0.0, -0.0, 1.0, -3.0, 1e-30]])
    cp = _f32_values(g, 9)
    cq = (np.abs(_f32_values(g, 5)) + 0.5).astype(np.float32).astype(np.float64)
    horner = orc.MapSpec("horner", cp)
    rational = orc.MapSpec("rational", cp[:7], cq)
    newton = orc.MapSpec("newton_cbrt", iters=6)

    def horner_rn(c, v):
        p = Fraction(c[-1])
        for ck in c[-2::-1]:
            p = Fraction(_rn32(p * Fraction(v) + Fraction(ck)))
        return p

    got_h = orc.map_values_f32(horner, x)
    got_r = orc.map_values_f32(rational, x)
    got_n = orc.map_values_f32(newton, x)
    for i, v in enumerate(x):
        assert got_h[i] == float(horner_rn(cp, v))
        assert got_r[i] == _rn32(horner_rn(cp[:7], v) / horner_rn(cq, v))
        y = Fraction(-1 if math.copysign(1.0, v) < 0 else 1)
        for _ in range(6):
            yy = Fraction(_rn32(y * y))
            q = Fraction(_rn32(Fraction(v) / yy))
            s = Fraction(_rn32(2 * y + q))
            y = Fraction(_rn32(s / 3))
        assert got_n[i] == float(y), (v, got_n[i], float(y))


def test_map_f32_matches_numpy_binary32(orc):
    """x^2 and P/Q with degree-0 polynomials are single binary32 operations:
    numpy's float32 arithmetic gives them independently."""
    g = np.random.default_rng(33)
    x = g.standard_normal(10_000).astype(np.float32)
    assert np.array_equal(orc.map_values_f32(orc.MapSpec("square"), x), (x * x).astype(np.float64))
    a, b = np.float32(1.7), g.uniform(0.5, 4.0, 10_000).astype(np.float32)
    got = np.array([orc.map_values_f32(orc.MapSpec("rational", [float(a)], [float(bb)]), [0.0])[0] for bb in b[:500]])
    assert np.array_equal(got, (a / b[:500]).astype(np.float64))


def test_reduce_mt_f32_values(orc):
    """With f32=True the threaded reductions sum the binary32 map values exactly."""
    g = np.random.default_rng(34)
    x = g.uniform(-2, 2, 20_001).astype(np.float32)
    m = orc.MapSpec("horner", _f32_values(g, 13))
    f = orc.map_values_f32(m, x)
    s, lo, hi, sa = orc.reduce_float_mt(m, x, 3, f32=True)
    assert s == math.fsum(f) and lo == f.min() and hi == f.max() and sa == math.fsum(np.abs(f))
    off = np.array([0, 5, 5, 9000, 20_001], dtype=np.int64)
    ss, sl, sh, sa = orc.segmented_reduce_float_mt(m, x, off, 2, f32=True)
    for k in range(4):
        seg = f[off[k]:off[k + 1]]
        assert ss[k] == math.fsum(seg) and sa[k] == math.fsum(np.abs(seg))
        if seg.size:
            assert sl[k] == seg.min() and sh[k] == seg.max()
