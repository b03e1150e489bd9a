"""The domain on which the vectorised Newton cube root runs without guards.

The device evaluates the map's steps y <- RN(RN(2y + RN(x / y^2)) / 3) from
y = 1 without checking the division's fast domain or the division by 3 when
every |x| of a lane lies in [2^-60, 2^28].  That rests on a bound: every
iterate stays within a few ulps of [min(1, c), max(1, (2 + x) / 3)] with
c = x^(1/3), so every divisor y^2 lies in [2^-42, 2^54] and every s RN(1/3)
is finite and at least 2^-22.  Here the binary32 steps are replayed on the
CPU (numpy float32 products and quotients, which are the IEEE operations;
the fused steps through FP64, whose extra rounding can move a result by an
ulp, far inside the margins checked) over a dense log-uniform sample of the
domain and its edges, for up to 64 steps, and every intermediate is checked
against those ranges.
"""
import numpy as np

F32 = np.float32
THIRD = F32(1.0) / F32(3.0)


def _domain_sample():
    g = np.random.default_rng(2028)
    lo, hi = F32(2.0 ** -60), F32(2.0 ** 28)
    x = np.exp2(g.uniform(-60.0, 28.0, 400_000)).astype(F32)
    edges = np.array([lo, hi, np.nextafter(lo, F32(1)), np.nextafter(hi, F32(0)), 1.0, 8.0, 27.0,
                      np.nextafter(F32(1), F32(0)), np.nextafter(F32(1), F32(2))], F32)
    x = np.concatenate([x, edges])
    return x[(x >= lo) & (x <= hi)]


def test_newton_iterates_stay_in_the_guard_free_ranges():
    x = _domain_sample()
    c = np.cbrt(x.astype(np.float64))
    y = np.ones_like(x)
    for step in range(64):
        b = (y * y).astype(F32)                                            # the divisor y^2
        assert np.all(b >= 2.0 ** -42) and np.all(b <= 2.0 ** 54), step
        q = (x / b).astype(F32)                                            # RN(x / y^2)
        s = (2.0 * y.astype(np.float64) + q.astype(np.float64)).astype(F32)  # fma(2, y, q)
        q0 = (s * THIRD).astype(F32)
        assert np.all(np.isfinite(q0)) and np.all(q0 >= 2.0 ** -22), step
        r = (s.astype(np.float64) - 3.0 * q0.astype(np.float64)).astype(F32)
        y = (r.astype(np.float64) * np.float64(THIRD) + q0.astype(np.float64)).astype(F32)
        lower = np.minimum(1.0, c) * (1.0 - 2.0 ** -20)
        upper = np.maximum(1.0, (2.0 + x.astype(np.float64)) / 3.0) * (1.0 + 2.0 ** -20)
        assert np.all(y >= lower) and np.all(y <= upper), step
        assert np.all(y >= 2.0 ** -21) and np.all(y <= 2.0 ** 27), step


def test_negative_inputs_mirror_exactly():
    """x < 0 runs the same steps on -x with every value negated (round to
    nearest is symmetric), so the bounds above cover it."""
    x = _domain_sample()[:50_000]
    yp, yn = np.ones_like(x), -np.ones_like(x)
    xn = -x
    for _ in range(8):
        for y, xx in ((yp, x), (yn, xn)):
            q = (xx / (y * y).astype(F32)).astype(F32)
            s = (2.0 * y.astype(np.float64) + q.astype(np.float64)).astype(F32)
            q0 = (s * THIRD).astype(F32)
            r = (s.astype(np.float64) - 3.0 * q0.astype(np.float64)).astype(F32)
            y[:] = (r.astype(np.float64) * np.float64(THIRD) + q0.astype(np.float64)).astype(F32)
        assert np.array_equal(yn.view(np.int32), (-yp).view(np.int32))
