"""tr_scan_reduce: the scan (inclusive or exclusive) and the sum / min / max of
the same f from one read of x, against the oracle.

Integer scans and their sums, minima and maxima are compared bit for bit;
float scans of x^2 >= 0 within 1e-5 relative per output (the scan's bar),
other float maps within the derived per-prefix bound of the parity tests;
float sums within 1e-6 normwise, float min / max within the map's error
bound.  The invariant scan[n-1] == sum (no carry-in) is checked bit for bit
for integers.  Sizes span one tile, many tiles and ragged tails; n = 0 gives
the identities.
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


def run(B, m, x, y_dtype, exclusive, carry=None, ops=7, sum_dtype=None, mm_dtype=torch.float32):
    n = x.numel()
    yt = B.dtype_of(torch.empty(0, dtype=y_dtype))
    ws = B.workspace(B.tr_scan_workspace_size(n, B.dtype_of(x), yt))
    y = torch.full((n,), 77, dtype=y_dtype, device="cuda")
    s = torch.full((1,), 99, dtype=sum_dtype or y_dtype, device="cuda")
    lo = torch.full((1,), 5, dtype=mm_dtype, device="cuda")
    hi = torch.full((1,), 5, dtype=mm_dtype, device="cuda")
    ex = B.make_exec(ws)
    B.tr_scan_reduce(m, x, y, ex, exclusive=exclusive, carry_in=carry, ops=ops, out_sum=s if ops & 1 else None,
                     out_min=lo if ops & 2 else None, out_max=hi if ops & 4 else None)
    B.tr_check(ex)
    return y, s, lo, hi


@pytest.mark.parametrize("kind", ["splitmix32", "xorshift32"])
@pytest.mark.parametrize("exclusive", [False, True], ids=["incl", "excl"])
@pytest.mark.parametrize("n", [1, 31, 8191, 8192, 8193, 100_003, 1 << 20])
def test_u32_bitexact(orc, B, kind, exclusive, n):
    x = I.u32(I.rng("misc", n + 3), n)
    xd = to_dev(x)
    spec = orc.MapSpec(kind)
    rs, rlo, rhi = orc.reduce_u32(spec, x)
    y, s, lo, hi = run(B, {"kind": kind}, xd, torch.int32, exclusive, mm_dtype=torch.int32)
    assert np.array_equal(u32_host(y), orc.scan_u32(spec, x, exclusive=exclusive))
    assert int(u32_host(s)[0]) == rs % (1 << 32)
    assert int(u32_host(lo)[0]) == rlo and int(u32_host(hi)[0]) == rhi
    y, s, lo, hi = run(B, {"kind": kind}, xd, torch.int64, exclusive, mm_dtype=torch.int32)
    assert np.array_equal(u64_host(y), orc.scan_u32_u64(spec, x, exclusive=exclusive))
    assert int(u64_host(s)[0]) == rs
    if not exclusive:
        assert int(u64_host(y)[-1]) == int(u64_host(s)[0])  # invariant: last prefix == sum
    assert int(u32_host(lo)[0]) == rlo and int(u32_host(hi)[0]) == rhi


def test_u32_carry_misaligned_and_partial_ops(orc, B):
    n = 50_001
    x = I.u32(I.rng("misc", 41), n)
    spec = orc.MapSpec("splitmix32")
    carry = torch.tensor([987654321], dtype=torch.int32, device="cuda")
    xd = to_dev(x, offset=1)
    y, s, _, hi = run(B, {"kind": "splitmix32"}, xd, torch.int32, True, carry=carry, ops=1 | 4,
                      mm_dtype=torch.int32)
    ref = (orc.scan_u32(spec, x, exclusive=True).astype(np.uint64) + 987654321).astype(np.uint32)
    assert np.array_equal(u32_host(y), ref)
    rs, _, rhi = orc.reduce_u32(spec, x)
    assert int(u32_host(s)[0]) == rs % (1 << 32)  # the sum leaves the carry out
    assert int(u32_host(hi)[0]) == rhi


@pytest.mark.parametrize("dt", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("exclusive", [False, True], ids=["incl", "excl"])
@pytest.mark.parametrize("n", [1, 4097, 100_003, 1 << 20])
def test_square_f32(orc, B, dt, exclusive, n):
    g = np.random.default_rng(n + 7)
    x64 = g.uniform(0, 1, n)
    if dt == "bf16":
        t = torch.from_numpy(x64).to(torch.bfloat16)
        xh = t.double().numpy()
    else:
        a = x64.astype(np.float32 if dt == "f32" else np.float16)
        t, xh = torch.from_numpy(a), a.astype(np.float64)
    m = I.simple_map("square")
    y, s, lo, hi = run(B, m, t.cuda(), torch.float32, exclusive, sum_dtype=torch.float64)
    spec = orc.MapSpec("square")
    ref = orc.scan_float(spec, xh, 24, exclusive=exclusive)
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-38)
    rs, rlo, rhi = orc.reduce_float(spec, xh)
    f = orc.map_values(spec, xh)
    bnd = map_error_bound(m, xh, f)
    assert abs(float(s.item()) - rs) <= 1e-6 * np.sum(np.abs(f)) + np.sum(bnd)
    assert abs(float(lo.item()) - rlo) <= bnd.max() + 2.0 ** -24 * abs(rlo)
    assert abs(float(hi.item()) - rhi) <= bnd.max() + 2.0 ** -24 * abs(rhi)


@pytest.mark.parametrize("mi", ["rational66", "newton6"])
def test_general_maps_exclusive(orc, B, mi):
    g = np.random.default_rng(8)
    if mi == "rational66":
        m = I.rational_map(I.f32_exact(g.standard_normal(7)), I.f32_exact(I.positive_even_q(g, 6)))
    else:
        m = I.newton_map(6)
    n = 200_001
    x = g.uniform(-2, 2, n).astype(np.float32)
    xh = x.astype(np.float64)
    y, s, lo, hi = run(B, m, torch.from_numpy(x).cuda(), torch.float32, True, sum_dtype=torch.float64)
    spec = oracle_map(orc, m)
    ref = orc.scan_float(spec, xh, 24, exclusive=True)
    f = orc.map_values(spec, xh)
    b = map_error_bound(m, xh, f)
    cf = np.concatenate([[0.0], np.cumsum(np.abs(f))[:-1]])
    cb = np.concatenate([[0.0], np.cumsum(b)[:-1]])
    got = y.cpu().double().numpy()
    assert np.all(np.abs(got - ref) <= 2.0 ** -23 * np.abs(ref) + 1e-6 * cf + cb)
    rs, rlo, rhi = orc.reduce_float(spec, xh)
    assert abs(float(s.item()) - rs) <= 1e-6 * np.sum(np.abs(f)) + np.sum(b)
    assert abs(float(lo.item()) - rlo) <= b.max() + 2.0 ** -24 * abs(rlo)
    assert abs(float(hi.item()) - rhi) <= b.max() + 2.0 ** -24 * abs(rhi)


def test_empty_gives_identities(B):
    x = torch.empty(0, dtype=torch.float32, device="cuda")
    y, s, lo, hi = run(B, I.simple_map("square"), x, torch.float32, False, sum_dtype=torch.float64)
    assert float(s.item()) == 0.0 and float(lo.item()) == np.inf and float(hi.item()) == -np.inf
    xu = torch.empty(0, dtype=torch.int32, device="cuda")
    y, s, lo, hi = run(B, {"kind": "splitmix32"}, xu, torch.int64, True, mm_dtype=torch.int32)
    assert int(s.item()) == 0 and int(u32_host(lo)[0]) == 0xFFFFFFFF and int(u32_host(hi)[0]) == 0


def test_nan_ignored_by_min_max(B):
    """min / max follow minNum / maxNum: NaN values are skipped."""
    x = torch.tensor([1.0, float("nan"), -3.0, 2.0] * 3000, dtype=torch.float32, device="cuda")
    _, _, lo, hi = run(B, I.simple_map("identity"), x, torch.float32, False, ops=6)
    assert float(lo.item()) == -3.0 and float(hi.item()) == 2.0


def test_same_as_separate_scan_and_reduce(B):
    """The fused pass gives the same scan bits as tr_scan and, for integers, the
    same sum as tr_reduce (bit for bit)."""
    n = 3_000_017
    xd = to_dev(I.u32(I.rng("misc", 77), n))
    y, s, _, _ = run(B, {"kind": "xorshift32"}, xd, torch.int64, False, ops=1)
    ws = B.workspace(B.tr_scan_workspace_size(n, B.TR_U32, B.TR_U64))
    y2 = torch.empty(n, dtype=torch.int64, device="cuda")
    ex = B.make_exec(ws)
    B.tr_scan({"kind": "xorshift32"}, xd, y2, ex)
    wr = B.workspace(B.tr_reduce_workspace_size(n, B.TR_U32))
    s2 = torch.zeros(1, dtype=torch.int64, device="cuda")
    exr = B.make_exec(wr)
    B.tr_reduce({"kind": "xorshift32"}, xd, 1, s2, None, None, exr)
    B.tr_check(ex)
    B.tr_check(exr)
    assert torch.equal(y, y2) and int(s.item()) == int(s2.item())


@pytest.mark.parametrize("exclusive", [False, True], ids=["incl", "excl"])
def test_scan_reduce_captured_in_a_cuda_graph(orc, B, exclusive):
    """The TMA-fed scan (a cooperative launch) with its fused reduction,
    captured into a CUDA graph and replayed twice: bit-exact outputs and
    reduction every time."""
    n = 1_000_003
    x = I.u32(I.rng("misc", 31), n)
    xd = to_dev(x)
    y = torch.empty(n, dtype=torch.int32, device="cuda")
    sm = torch.zeros(1, dtype=torch.int32, device="cuda")
    lo = torch.zeros(1, dtype=torch.int32, device="cuda")
    hi = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = B.workspace(B.tr_scan_workspace_size(n, B.TR_U32, B.TR_U32))
    spec = orc.MapSpec("splitmix32")
    ref = orc.scan_u32(spec, x, exclusive=exclusive)
    rs, rlo, rhi = orc.reduce_u32(spec, x)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            ex = B.make_exec(ws)
            B.tr_scan_reduce({"kind": "splitmix32"}, xd, y, ex, exclusive=exclusive, ops=7, out_sum=sm, out_min=lo,
                             out_max=hi)
    for _ in range(2):
        y.fill_(-1)
        sm.zero_()
        torch.cuda.synchronize()
        g.replay()
        torch.cuda.synchronize()
        assert np.array_equal(u32_host(y), ref)
        assert int(u32_host(sm)[0]) == rs % (1 << 32)
        assert int(u32_host(lo)[0]) == rlo and int(u32_host(hi)[0]) == rhi
    B.tr_check(B.make_exec(ws))
