"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integers and integer scans are compared bit for bit; FP64 maps bit for bit;
FP32-compute results within bounds derived from the arithmetic (see
tests/helpers.py): the per-element map error bound plus a summation term of
1e-6 * sum |f| for compensated sums and scans.  Sizes span several tiles,
ragged tails, tiny and empty inputs, and misaligned base pointers.
"""
import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import map_error_bound, oracle_map, to_dev, u32_host, u64_host

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


SIZES = [0, 1, 5, 31, 32, 33, 127, 4095, 4096, 4097, 65537, 1_000_003]
NPDT = {"f16": np.float16, "f32": np.float32}


def _float_maps(rng):
    return [
        I.simple_map("identity"),
        I.simple_map("square"),
        I.horner_map(I.f32_exact(rng.standard_normal(9))),       # degree 8: register-resident form
        I.horner_map(I.f32_exact(rng.standard_normal(12))),      # degree 11: run-time form
        I.rational_map(I.f32_exact(rng.standard_normal(7)), I.f32_exact(I.positive_even_q(rng, 6))),
        I.rational_map(I.f32_exact(rng.standard_normal(4)), I.f32_exact(I.positive_even_q(rng, 4))),
        I.newton_map(6),
    ]


MAPS = _float_maps(np.random.default_rng(77))
MAP_IDS = ["identity", "square", "horner8", "horner11", "rational66", "rational34", "newton6"]


def host_input(dt, n, seed, lo=-2.0, hi=2.0):
    """(CPU tensor in storage dtype, its exact FP64 values)."""
    g = np.random.default_rng(seed)
    x64 = g.uniform(lo, hi, n)
    if dt == "bf16":
        t = torch.from_numpy(x64).to(torch.bfloat16)
        return t, t.double().numpy()
    a = x64.astype(NPDT[dt])
    return torch.from_numpy(a), a.astype(np.float64)


def dev(t, offset=0):
    if offset:
        buf = torch.empty(t.numel() + offset, dtype=t.dtype, device="cuda")
        buf[offset:].copy_(t.cuda())
        return buf[offset:]
    return t.cuda()


# ----------------------------------------------------------------------------- map

@pytest.mark.parametrize("mi", range(len(MAPS)), ids=MAP_IDS)
@pytest.mark.parametrize("dt", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("n,off", [(1, 0), (33, 0), (4097, 0), (100_003, 0), (100_003, 1), (4099, 3)])
def test_map_float(orc, B, mi, dt, n, off):
    m = MAPS[mi]
    th, xh = host_input(dt, n, seed=n + mi)
    x = dev(th, off)
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    B.tr_map(m, x, y)
    ref = orc.map_values(oracle_map(orc, m), xh)
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= map_error_bound(m, xh, ref)), np.max(np.abs(got - ref))
    # the same sequence in binary32: bit for bit
    assert np.array_equal(got.view(np.int64), orc.map_values_f32(oracle_map(orc, m), xh).view(np.int64))


def _newton_magnitude_mix(seed: int) -> np.ndarray:
    """Groups of four consecutive f32 values (one 16-byte vector, the map
    kernel's unit): groups wholly inside [2^-60, 2^28] in magnitude (the Newton
    map's guard-free steps), groups on and just inside those edges, and groups
    holding one value outside them (zeros, subnormals, tiny, huge, infinities,
    NaN, and the edges' outer neighbours), which take the guarded steps."""
    g = np.random.default_rng(seed)
    f32 = np.float32

    def signed(mag):
        return (mag * np.where(g.random(mag.size) < 0.5, -1.0, 1.0)).astype(f32)

    inside = signed(np.exp2(g.uniform(-60, 28, 4 * 20000)))
    lo, hi = f32(2.0 ** -60), f32(2.0 ** 28)
    edge_in = np.array([lo, hi, np.nextafter(lo, f32(1)), np.nextafter(hi, f32(0))], f32)
    edges = signed(np.resize(edge_in, 4 * 500).astype(np.float64))
    outer = np.array([0.0, -0.0, 1e-45, -1e-45, 1.17549435e-38, 2.0 ** -100, 2.0 ** 40, 3.4028235e38, np.inf,
                      -np.inf, np.nan, np.nextafter(lo, f32(0)), np.nextafter(hi, f32(np.inf)), 2.0 ** -61],
                     f32)
    mixed = signed(np.exp2(g.uniform(-60, 28, 4 * 3000))).reshape(-1, 4)
    mixed[np.arange(mixed.shape[0]), g.integers(0, 4, mixed.shape[0])] = g.choice(outer, mixed.shape[0])
    wide = signed(np.exp2(g.uniform(-149, 127, 4 * 5000)))
    groups = np.concatenate([inside.reshape(-1, 4), edges.reshape(-1, 4), mixed, wide.reshape(-1, 4)])
    return groups[g.permutation(groups.shape[0])].ravel()


@pytest.mark.parametrize("iters", [6, 40])
def test_newton_all_magnitudes_bitexact(orc, B, iters):
    """The Newton cube root runs without its guards when every value of a
    vector lies in [2^-60, 2^28] in magnitude: over values of every magnitude,
    the edges and the special values, the map equals the oracle's binary32
    evaluation bit for bit (NaN as NaN), and a reduction over the guard-free
    values gives the oracle's minimum and maximum exactly."""
    m = I.newton_map(iters)
    xh = _newton_magnitude_mix(500 + iters)
    y = torch.empty(xh.size, dtype=torch.float32, device="cuda")
    B.tr_map(m, torch.from_numpy(xh).cuda(), y)
    got = y.cpu().numpy()
    ref = orc.map_values_f32(oracle_map(orc, m), xh.astype(np.float64)).astype(np.float32)
    same = (got.view(np.int32) == ref.view(np.int32)) | (np.isnan(got) & np.isnan(ref))
    assert np.all(same), (xh[~same][:8], got[~same][:8], ref[~same][:8])
    fin = xh[(np.abs(xh) >= 2.0 ** -60) & (np.abs(xh) <= 2.0 ** 28)]
    s, lo, hi = reduce_dev(B, m, torch.from_numpy(fin).cuda())
    f = orc.map_values_f32(oracle_map(orc, m), fin.astype(np.float64))
    assert lo == np.min(f) and hi == np.max(f)
    assert abs(s - np.sum(f.astype(np.float64))) <= 1e-6 * np.sum(np.abs(f))


def test_rational_all_magnitudes_bitexact(orc, B):
    """The rational map over inputs of every magnitude (groups of four inside
    [-512, 512], groups far outside it, values next to the numerator's real
    roots, and the special values): the division-free quotient where the
    guard admits it, the IEEE division elsewhere, and the map equals the
    oracle's binary32 evaluation bit for bit."""
    g = np.random.default_rng(2309)
    cp = I.f32_exact(g.standard_normal(7))
    m = I.rational_map(cp, I.f32_exact(I.positive_even_q(g, 6)))
    f32 = np.float32
    inside = g.uniform(-512, 512, 4 * 20000)
    roots = np.roots(np.asarray(cp, np.float64)[::-1])
    roots = roots[np.abs(roots.imag) < 1e-12].real
    near = np.concatenate([[np.nextafter(f32(r), f32(d * np.inf)) for d in (-1, 1) for _ in range(2)] for r in roots]
                          + [np.zeros(0)])
    outside = g.choice([-1.0, 1.0], 4 * 5000) * np.exp2(g.uniform(-149, 127, 4 * 5000))
    special = np.array([0.0, -0.0, 1e-45, np.inf, -np.inf, np.nan, 512.0, -512.0, 512.00006, 3.4028235e38], f32)
    groups = [inside.astype(f32).reshape(-1, 4), outside.astype(f32).reshape(-1, 4),
              np.resize(np.concatenate([near, special]).astype(f32), 4 * 200).reshape(-1, 4)]
    mixed = g.uniform(-2, 2, 4 * 2000).astype(f32).reshape(-1, 4)
    mixed[:, 0] = g.choice(np.concatenate([special, near.astype(f32)]), mixed.shape[0])
    groups.append(mixed)
    x = np.concatenate(groups)
    x = x[g.permutation(x.shape[0])].ravel()
    y = torch.empty(x.size, dtype=torch.float32, device="cuda")
    B.tr_map(m, torch.from_numpy(x).cuda(), y)
    got = y.cpu().numpy()
    ref = orc.map_values_f32(oracle_map(orc, m), x.astype(np.float64)).astype(np.float32)
    same = (got.view(np.int32) == ref.view(np.int32)) | (np.isnan(got) & np.isnan(ref))
    assert np.all(same), (x[~same][:8], got[~same][:8], ref[~same][:8])
    # the reduce kernel's 16-value groups on the same values: min / max exact
    s, lo, hi = reduce_dev(B, m, torch.from_numpy(x[np.isfinite(x) & (np.abs(x) <= 512)]).cuda())
    f = orc.map_values_f32(oracle_map(orc, m), x[np.isfinite(x) & (np.abs(x) <= 512)].astype(np.float64))
    assert lo == np.min(f) and hi == np.max(f)


@pytest.mark.parametrize("deg", [0, 1, 3, 5, 13, 16, 17, 24])
def test_horner_runtime_degrees(orc, B, deg):
    """Horner maps of run-time degree (packed up to degree 16, the coefficient
    loop above): map bit for bit against the binary32 oracle map; reduce within
    1e-6 of the exact sum of those values, min / max exact."""
    g = np.random.default_rng(300 + deg)
    m = I.horner_map(I.f32_exact(g.standard_normal(deg + 1) / (np.arange(deg + 1) + 1.0)))
    n = 100_003
    xh = g.uniform(-1.2, 1.2, n).astype(np.float32)
    x = torch.from_numpy(xh).cuda()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    B.tr_map(m, x, y)
    f32 = orc.map_values_f32(oracle_map(orc, m), xh)
    assert np.array_equal(y.cpu().double().numpy().view(np.int64), f32.view(np.int64))
    s, lo, hi = reduce_dev(B, m, x)
    rs, rlo, rhi, ra = orc.reduce_float_mt(oracle_map(orc, m), xh, f32=True)
    assert abs(s - rs) <= 1e-6 * ra and lo == rlo and hi == rhi


@pytest.mark.parametrize("mi", range(len(MAPS)), ids=MAP_IDS)
def test_map_f64_bitexact(orc, B, mi):
    """FP64 device evaluation = FP64 oracle, bit for bit (same fma/division sequence)."""
    m = MAPS[mi]
    x = np.random.default_rng(5).uniform(-2, 2, 50_001)
    y = torch.empty(x.size, dtype=torch.float64, device="cuda")
    B.tr_map(m, torch.from_numpy(x).cuda(), y)
    ref = orc.map_values(oracle_map(orc, m), x)
    assert np.array_equal(y.cpu().numpy().view(np.int64), ref.view(np.int64))


@pytest.mark.parametrize("kind", ["xorshift32", "splitmix32", "identity"])
@pytest.mark.parametrize("n,off", [(1, 0), (4097, 0), (1_000_003, 0), (4099, 1)])
def test_map_u32_bitexact(orc, B, kind, n, off):
    x = I.u32(I.rng("misc", n), n)
    xd = to_dev(x, offset=off)
    y = torch.empty(n, dtype=torch.int32, device="cuda")
    B.tr_map({"kind": kind}, xd, y)
    assert np.array_equal(u32_host(y), orc.map_values(orc.MapSpec(kind), x))


def test_map_inplace(orc, B):
    x = np.random.default_rng(9).uniform(-1, 1, 10_000).astype(np.float32)
    t = torch.from_numpy(x).cuda()
    m = MAPS[2]
    B.tr_map(m, t, t)
    xd = x.astype(np.float64)
    ref = orc.map_values(oracle_map(orc, m), xd)
    assert np.all(np.abs(t.cpu().double().numpy() - ref) <= map_error_bound(m, xd, ref))


@pytest.fixture(scope="module")
def host_bin():
    from tests.test_hdc import build_host_check
    return build_host_check()


@pytest.mark.parametrize("mi", range(len(MAPS)), ids=MAP_IDS)
def test_map_fp32_device_equals_host_build(B, host_bin, mi):
    """hdc: the device build of maps.h and the g++ host build give the same bits."""
    from tests.test_hdc import host_eval
    m = MAPS[mi]
    x = np.random.default_rng(10).uniform(-2, 2, 20_000).astype(np.float32)
    y = torch.empty(x.size, dtype=torch.float32, device="cuda")
    B.tr_map(m, torch.from_numpy(x).cuda(), y)
    host = host_eval(host_bin, m, x.astype(np.float64), "f").astype(np.float32)
    assert np.array_equal(y.cpu().numpy().view(np.int32), host.view(np.int32))


# -------------------------------------------------------------------------- reduce

def reduce_dev(B, m, x, sum_dtype=torch.float64, mm_dtype=torch.float32):
    n = x.numel()
    ws = B.workspace(B.tr_reduce_workspace_size(n, B.dtype_of(x)))
    s = torch.full((1,), 7.0, dtype=sum_dtype, device="cuda")
    lo = torch.zeros(1, dtype=mm_dtype, device="cuda")
    hi = torch.zeros(1, dtype=mm_dtype, device="cuda")
    ex = B.make_exec(ws)
    B.tr_reduce(m, x, B.TR_SUM | B.TR_MIN | B.TR_MAX, s, lo, hi, ex)
    B.tr_check(ex)
    return s.cpu().double().item(), lo.cpu().double().item(), hi.cpu().double().item()


def check_float_reduce(orc, m, xh, got, sum_f32=False):
    ref = orc.map_values(oracle_map(orc, m), xh)
    s_ref, lo_ref, hi_ref = orc.reduce_float(oracle_map(orc, m), xh)
    bnd = map_error_bound(m, xh, ref)
    tol = 1e-6 * np.sum(np.abs(ref)) + np.sum(bnd) + (abs(s_ref) * 2.0 ** -24 if sum_f32 else 0.0) + 1e-30
    s, lo, hi = got
    assert abs(s - s_ref) <= tol, (s, s_ref, tol)
    if xh.size:
        mb = np.max(bnd) + 2.0 ** -24 * max(abs(lo_ref), abs(hi_ref))
        assert abs(lo - lo_ref) <= mb and abs(hi - hi_ref) <= mb
        # against the binary32 map values: the compensated sum within 1e-6 normwise, min / max exact
        s32, lo32, hi32, a32 = orc.reduce_float_mt(oracle_map(orc, m), xh, 1, f32=True)
        assert abs(s - s32) <= 1e-6 * a32 + (abs(s32) * 2.0 ** -24 if sum_f32 else 0.0), (s, s32, a32)
        assert lo == lo32 and hi == hi32
    else:
        assert s == 0.0 and lo == np.inf and hi == -np.inf


@pytest.mark.parametrize("mi", range(len(MAPS)), ids=MAP_IDS)
@pytest.mark.parametrize("dt", ["f16", "bf16", "f32"])
@pytest.mark.parametrize("n", SIZES)
def test_reduce_float(orc, B, mi, dt, n):
    m = MAPS[mi]
    th, xh = host_input(dt, n, seed=3 * n + mi)
    check_float_reduce(orc, m, xh, reduce_dev(B, m, th.cuda()))


@pytest.mark.parametrize("off", [1, 2, 3, 5])
def test_reduce_misaligned(orc, B, off):
    m = MAPS[4]
    th, xh = host_input("f32", 70_001, seed=off)
    check_float_reduce(orc, m, xh, reduce_dev(B, m, dev(th, off)))
    th, xh = host_input("f16", 70_001, seed=off)
    check_float_reduce(orc, m, xh, reduce_dev(B, m, dev(th, off)))


def test_reduce_f32_sum_output(orc, B):
    m = MAPS[2]
    th, xh = host_input("f32", 300_000, seed=1)
    check_float_reduce(orc, m, xh, reduce_dev(B, m, th.cuda(), sum_dtype=torch.float32), sum_f32=True)


@pytest.mark.parametrize("n", [0, 1, 3, 4097, 1 << 20])
def test_reduce_f64_horner(orc, B, n):
    """FP64 path: min / max bit-exact (same fma sequence), sum normwise <= 1e-13."""
    x, m = I.horner_f64(n)
    s, lo, hi = reduce_dev(B, m, torch.from_numpy(x).cuda(), mm_dtype=torch.float64)
    s_ref, lo_ref, hi_ref = orc.reduce_float(oracle_map(orc, m), x)
    f = orc.map_values(oracle_map(orc, m), x)
    assert lo == lo_ref and hi == hi_ref
    assert abs(s - s_ref) <= 1e-13 * np.sum(np.abs(f)) or (n == 0 and s == 0.0)


@pytest.mark.parametrize("kind", ["xorshift32", "splitmix32", "identity"])
@pytest.mark.parametrize("n,off", [(0, 0), (1, 0), (33, 0), (4097, 0), (1 << 20, 0), (1_000_003, 3)])
def test_reduce_u32_bitexact(orc, B, kind, n, off):
    x = I.u32(I.rng("misc", n + 1), n)
    xd = to_dev(x, offset=off)
    ws = B.workspace(B.tr_reduce_workspace_size(n, B.TR_U32))
    s = torch.zeros(1, dtype=torch.int64, device="cuda")
    s32 = torch.zeros(1, dtype=torch.int32, device="cuda")
    lo = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi = torch.zeros(1, dtype=torch.int32, device="cuda")
    ex = B.make_exec(ws)
    B.tr_reduce({"kind": kind}, xd, B.TR_SUM | B.TR_MIN | B.TR_MAX, s, lo, hi, ex)
    B.tr_reduce({"kind": kind}, xd, B.TR_SUM, s32, None, None, ex)
    B.tr_check(ex)
    rs, rlo, rhi = orc.reduce_u32(orc.MapSpec(kind), x)
    assert int(u64_host(s)[0]) == rs
    assert int(u32_host(s32)[0]) == rs % (1 << 32)
    assert int(u32_host(lo)[0]) == rlo and int(u32_host(hi)[0]) == rhi


def test_reduce_deterministic(B):
    m = MAPS[4]
    th, _ = host_input("f32", 2_000_003, seed=4)
    x = th.cuda()
    a = reduce_dev(B, m, x)
    for _ in range(3):
        assert reduce_dev(B, m, x) == a


# ---------------------------------------------------------------------------- scan

def scan_dev(B, m, x, yt_torch, carry=None, out=None):
    n = x.numel()
    yt = B.dtype_of(torch.empty(0, dtype=yt_torch))
    ws = B.workspace(B.tr_scan_workspace_size(n, B.dtype_of(x), yt))
    y = out if out is not None else torch.empty(n, dtype=yt_torch, device="cuda")
    ex = B.make_exec(ws)
    B.tr_scan(m, x, y, ex, carry_in=carry)
    B.tr_check(ex)
    return y


@pytest.mark.parametrize("kind", ["splitmix32", "xorshift32", "identity"])
@pytest.mark.parametrize("n,off", [(1, 0), (31, 0), (4095, 0), (4097, 0), (8191, 0), (8192, 0), (8193, 0),
                                   (24577, 0), (1 << 20, 0), (1_000_003, 0), (100_001, 1), (8193, 2)])
def test_scan_u32_bitexact(orc, B, kind, n, off):
    x = I.u32(I.rng("mixer_u32_scan", n), n)
    xd = to_dev(x, offset=off)
    y = scan_dev(B, {"kind": kind}, xd, torch.int32)
    assert np.array_equal(u32_host(y), orc.scan_u32(orc.MapSpec(kind), x))
    y64 = scan_dev(B, {"kind": kind}, xd, torch.int64)
    assert np.array_equal(u64_host(y64), orc.scan_u32_u64(orc.MapSpec(kind), x))


def test_scan_u32_carry_and_inplace(orc, B):
    n = 50_000
    x = I.u32(I.rng("misc", 5), n)
    ref = orc.scan_u32(orc.MapSpec("splitmix32"), x)
    carry = torch.tensor([123456789], dtype=torch.int32, device="cuda")
    xd = to_dev(x)
    y = scan_dev(B, {"kind": "splitmix32"}, xd, torch.int32, carry=carry)
    assert np.array_equal(u32_host(y), (ref.astype(np.uint64) + 123456789).astype(np.uint32))
    scan_dev(B, {"kind": "splitmix32"}, xd, torch.int32, out=xd)  # in place
    assert np.array_equal(u32_host(xd), ref)


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("n,off", [(1, 0), (4095, 0), (4097, 0), (100_003, 0), (1 << 20, 0), (20_001, 1)])
def test_scan_square_f32(orc, B, dt, n, off):
    """x ~ U[0,1], f = x^2 >= 0: every prefix within 1e-5 relative."""
    th, xh = host_input(dt, n, seed=n, lo=0.0, hi=1.0)
    y = scan_dev(B, I.simple_map("square"), dev(th, off), torch.float32)
    ref = orc.scan_float(orc.MapSpec("square"), xh, 24)
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-38)


@pytest.mark.parametrize("mi", [2, 3, 4, 6], ids=["horner8", "horner11", "rational66", "newton6"])
def test_scan_general_sign(orc, B, mi):
    """Mixed-sign f: |y_i - ref_i| <= 2^-23 |ref_i| + 1e-6 sum_{j<=i} |f_j| + sum_{j<=i} bound_j."""
    m = MAPS[mi]
    th, xh = host_input("f32", 200_001, seed=mi)
    y = scan_dev(B, m, th.cuda(), torch.float32).cpu().double().numpy()
    ref = orc.scan_float(oracle_map(orc, m), xh, 24)
    f = orc.map_values(oracle_map(orc, m), xh)
    tol = 2.0 ** -23 * np.abs(ref) + 1e-6 * np.cumsum(np.abs(f)) + np.cumsum(map_error_bound(m, xh, f))
    assert np.all(np.abs(y - ref) <= tol)


def test_scan_telescoping_f32(B):
    """P = 1, Q = x^2 + x at x = 1..n: prefixes are 1 - 1/(k+1) (closed form)."""
    n = 300_000
    x = np.arange(1, n + 1, dtype=np.float32)
    y = scan_dev(B, I.rational_map([1.0], [0.0, 1.0, 1.0]), torch.from_numpy(x).cuda(), torch.float32)
    ref = 1 - 1 / (np.arange(1, n + 1) + 1.0)
    assert np.all(np.abs(y.cpu().double().numpy() - ref) <= 4 * 2.0 ** -24 * ref)


def test_scan_last_equals_reduce(B):
    """Invariant: scan[n-1] == reduce (bit exact for u32 mod 2^32)."""
    n = 3_000_001
    x = to_dev(I.u32(I.rng("misc", 9), n))
    y = scan_dev(B, {"kind": "xorshift32"}, x, torch.int32)
    ws = B.workspace(B.tr_reduce_workspace_size(n, B.TR_U32))
    s = torch.zeros(1, dtype=torch.int32, device="cuda")
    ex = B.make_exec(ws)
    B.tr_reduce({"kind": "xorshift32"}, x, B.TR_SUM, s, None, None, ex)
    B.tr_check(ex)
    assert u32_host(y)[-1] == u32_host(s)[0]


def test_scan_timeout_reports_and_recovers(orc, B):
    """A tile that never publishes makes its successor's bounded wait run out:
    tr_check reports TR_ERR_TIMEOUT, the context stays usable, and a
    re-initialised workspace scans correctly.  No trap, no hang."""
    n = 64 * 8192
    x = I.u32(I.rng("misc", 11), n)
    xd = to_dev(x)
    ws = B.workspace(B.tr_scan_workspace_size(n, B.TR_U32, B.TR_U32))
    y = torch.empty(n, dtype=torch.int32, device="cuda")
    ex = B.make_exec(ws, wait_timeout_us=20_000, debug_stall_tile=5)
    B.tr_scan({"kind": "splitmix32"}, xd, y, ex)
    with pytest.raises(B.TrError) as e:
        B.tr_check(ex)
    assert e.value.status == 6
    B.tr_workspace_init(ws)
    ex = B.make_exec(ws)
    B.tr_scan({"kind": "splitmix32"}, xd, y, ex)
    B.tr_check(ex)
    assert np.array_equal(u32_host(y), orc.scan_u32(orc.MapSpec("splitmix32"), x))


# --------------------------------------------------------------- segmented reduce

def segreduce_dev(B, m, x, off_np, sum_dtype=torch.float64):
    n = x.numel()
    nseg = off_np.size - 1
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, nseg, B.dtype_of(x)))
    off = torch.from_numpy(np.ascontiguousarray(off_np, dtype=np.int64)).cuda()
    sums = torch.full((nseg,), 7.0, dtype=sum_dtype, device="cuda")
    mins = torch.zeros(nseg, dtype=torch.float32, device="cuda")
    maxs = torch.zeros(nseg, dtype=torch.float32, device="cuda")
    ex = B.make_exec(ws)
    B.tr_segmented_reduce(m, x, off, B.TR_SUM | B.TR_MIN | B.TR_MAX, sums, mins, maxs, ex)
    B.tr_check(ex)
    return sums.cpu().double().numpy(), mins.cpu().double().numpy(), maxs.cpu().double().numpy()


def check_seg(orc, m, xh, off, got):
    s, lo, hi = got
    rs, rlo, rhi = orc.segmented_reduce_float(oracle_map(orc, m), xh, off)
    f = orc.map_values(oracle_map(orc, m), xh)
    b = map_error_bound(m, xh, f)
    cf = np.concatenate([[0.0], np.cumsum(np.abs(f))])
    cb = np.concatenate([[0.0], np.cumsum(b)])
    tol = 1e-6 * (cf[off[1:]] - cf[off[:-1]]) + (cb[off[1:]] - cb[off[:-1]]) + 1e-30
    assert np.all(np.abs(s - rs) <= tol), np.max(np.abs(s - rs) / tol)
    empty = off[1:] == off[:-1]
    assert np.all(np.isposinf(lo[empty])) and np.all(np.isneginf(hi[empty])) and np.all(s[empty] == 0)
    ne = ~empty
    mb = b.max() if b.size else 0.0
    assert np.all(np.abs(lo[ne] - rlo[ne]) <= mb + 2.0 ** -24 * np.abs(rlo[ne]))
    assert np.all(np.abs(hi[ne] - rhi[ne]) <= mb + 2.0 ** -24 * np.abs(rhi[ne]))
    # against the binary32 map values: compensated sums within 1e-6 normwise, min / max exact
    s32, lo32, hi32, a32 = orc.segmented_reduce_float_mt(oracle_map(orc, m), xh, off, f32=True)
    assert np.all(np.abs(s - s32) <= 1e-6 * a32), np.max(np.abs(s - s32) / np.maximum(a32, 1e-300))
    assert np.array_equal(lo[ne], lo32[ne]) and np.array_equal(hi[ne], hi32[ne])


def offsets_random(n, nseg, seed, max_len=8192):
    return I.segment_offsets(np.random.default_rng(seed), n, nseg, max_len)


@pytest.mark.parametrize("mi", range(len(MAPS)), ids=MAP_IDS)
@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
def test_segreduce_random(orc, B, mi, dt):
    m = MAPS[mi]
    n = 1_000_003
    off = offsets_random(n, 300, seed=mi)
    th, xh = host_input(dt, n, seed=mi + 50)
    check_seg(orc, m, xh, off, segreduce_dev(B, m, th.cuda(), off))


def test_segreduce_edge_structures(orc, B):
    m = MAPS[4]
    n = 200_000
    th, xh = host_input("f32", n, seed=99)
    x = th.cuda()
    cases = [
        np.array([0, n]),                                                  # one segment
        np.array([0, 0, 0, n, n, n]),                                      # empty segments at both ends
        np.concatenate([np.arange(0, 5001), [n]]),                         # 5000 length-1, then one long
        np.linspace(0, n, 7).astype(np.int64),                             # few long segments (cross warps)
        np.concatenate([[0], np.sort(np.random.default_rng(1).integers(0, n, 20000)), [n]]),  # many short/empty
    ]
    for off in cases:
        off = np.asarray(off, dtype=np.int64)
        check_seg(orc, m, xh, off, segreduce_dev(B, m, x, off))
    got = segreduce_dev(B, m, x[:0], np.zeros(4, dtype=np.int64))  # n = 0, all segments empty
    assert np.all(got[0] == 0) and np.all(np.isposinf(got[1])) and np.all(np.isneginf(got[2]))
    xm = dev(th[:n - 3], 3)  # misaligned base
    off = offsets_random(n - 3, 50, seed=3)
    check_seg(orc, m, xh[:n - 3], off, segreduce_dev(B, m, xm, off))


def test_segreduce_sum_of_segments_is_total(orc, B):
    m = MAPS[2]
    n = 500_000
    th, xh = host_input("f32", n, seed=5)
    off = offsets_random(n, 100, seed=5)
    s, _, _ = segreduce_dev(B, m, th.cuda(), off)
    tot, _, _ = reduce_dev(B, m, th.cuda())
    f = orc.map_values(oracle_map(orc, m), xh)
    assert abs(np.sum(s) - tot) <= 2e-6 * np.sum(np.abs(f)) + 2 * np.sum(map_error_bound(m, xh, f))


def test_segreduce_deterministic(B):
    m = MAPS[4]
    n = 3_000_000
    th, _ = host_input("f32", n, seed=6)
    off = offsets_random(n, 1000, seed=6)
    x = th.cuda()
    a = segreduce_dev(B, m, x, off)
    b = segreduce_dev(B, m, x, off)
    assert all(np.array_equal(u, v) for u, v in zip(a, b))


def test_segreduce_bad_offsets_reported(B):
    m = MAPS[4]
    n = 10_000
    x = torch.zeros(n, dtype=torch.float32, device="cuda")
    off = torch.tensor([0, 5000, 3000, n], dtype=torch.int64, device="cuda")  # not monotone
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, 3, B.TR_F32))
    sums = torch.zeros(3, dtype=torch.float64, device="cuda")
    ex = B.make_exec(ws)
    B.tr_segmented_reduce(m, x, off, B.TR_SUM, sums, None, None, ex)
    with pytest.raises(B.TrError) as e:
        B.tr_check(ex)
    assert e.value.status == 7


@pytest.mark.parametrize("dt", ["f32", "f16"])
def test_segreduce_boundaries_on_chunk_and_range_edges(orc, B, dt):
    """Segment ends placed exactly on (and one off) the 2 KiB streaming-chunk
    edges and on multiples of the per-warp range quantum, plus runs of empty
    segments sitting on those edges."""
    m = MAPS[4]
    n = (1 << 22) + 77
    th, xh = host_input(dt, n, seed=123)
    V = 4 if dt == "f32" else 8
    edges = set()
    for q in (128 * V, 32 * V * 14, 32 * V * 56):
        for k in range(1, n // q, 7):
            for d in (-1, 0, 1):
                edges.add(k * q + d)
    edges = sorted(e for e in edges if 0 < e < n)
    off = np.concatenate([[0], edges, edges[::50], [n, n]]).astype(np.int64)
    off.sort()
    check_seg(orc, m, xh, off, segreduce_dev(B, m, th.cuda(), off))


@pytest.mark.parametrize("misaligned", [False, True], ids=["tma", "unaligned"])
@pytest.mark.parametrize("case", ["first_not_zero", "last_not_n"])
def test_segreduce_offset_ends_reported(orc, B, misaligned, case):
    """Offsets whose ends break the contract (off[0] = 0, off[n_seg] = n) are
    reported as TR_ERR_DEVICE_ASSERT by tr_check on both walks (the TMA ring for
    16-byte aligned x, plain loads otherwise), and a valid call afterwards on a
    re-initialised workspace is exact again."""
    n = 1_000_000
    th, xh = host_input("f32", n, seed=31)
    x = dev(th, 1) if misaligned else th.cuda()
    off = np.linspace(0, n, 201).astype(np.int64)
    bad = off.copy()
    if case == "first_not_zero":
        bad[0] = 5000
    else:
        bad[-1] = n - 100
    m = MAPS[4]
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, 200, B.TR_F32))
    sums = torch.zeros(200, dtype=torch.float64, device="cuda")
    ex = B.make_exec(ws)
    B.tr_segmented_reduce(m, x, torch.from_numpy(bad).cuda(), B.TR_SUM, sums, None, None, ex)
    with pytest.raises(B.TrError) as e:
        B.tr_check(ex)
    assert e.value.status == 7
    B.tr_workspace_init(ws)
    check_seg(orc, m, xh, off, segreduce_dev(B, m, x, off))


def test_segreduce_host_buffers_equal_device_call(B):
    """tr_segmented_reduce_host (host buffers in and out, the copies enqueued by
    the call) gives the device call's results bit for bit, from page-locked and
    from pageable host memory; missing buffers are argument errors."""
    import ctypes
    m = MAPS[4]
    n = 3_000_017
    th, _ = host_input("f32", n, seed=41)
    off = offsets_random(n, 500, seed=41)
    nseg = off.size - 1
    ref = segreduce_dev(B, m, th.cuda(), off)
    L = B.lib()
    md = B.MapDesc(m)
    xd = torch.empty(n, dtype=torch.float32, device="cuda")
    offd = torch.empty(nseg + 1, dtype=torch.int64, device="cuda")
    sd = torch.empty(nseg, dtype=torch.float64, device="cuda")
    lod = torch.empty(nseg, dtype=torch.float32, device="cuda")
    hid = torch.empty(nseg, dtype=torch.float32, device="cuda")
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, nseg, B.TR_F32))
    ex = B.make_exec(ws)
    for pinned in (True, False):
        xh = th.pin_memory() if pinned else th.clone()
        offh = torch.from_numpy(off).pin_memory() if pinned else torch.from_numpy(off.copy())
        outs = [torch.zeros(nseg, dtype=dt) for dt in (torch.float64, torch.float32, torch.float32)]
        if pinned:
            outs = [o.pin_memory() for o in outs]
        st = L.tr_segmented_reduce_host(md.ref(), xh.data_ptr(), B.TR_F32, n, offh.data_ptr(), nseg, 7,
                                        outs[0].data_ptr(), B.TR_F64, outs[1].data_ptr(), outs[2].data_ptr(),
                                        xd.data_ptr(), offd.data_ptr(), sd.data_ptr(), lod.data_ptr(), hid.data_ptr(),
                                        ctypes.byref(ex))
        assert st == 0, L.tr_last_error()
        B.tr_check(ex)
        for got, want in zip(outs, ref):
            assert np.array_equal(got.double().numpy(), want)
    st = L.tr_segmented_reduce_host(md.ref(), th.data_ptr(), B.TR_F32, n, None, nseg, 7, None, B.TR_F64, None,
                                    None, xd.data_ptr(), offd.data_ptr(), sd.data_ptr(), lod.data_ptr(),
                                    hid.data_ptr(), ctypes.byref(ex))
    assert st == 1
