"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, against the oracle on outputs it can afford:

  * segmented rational 6/6, 2^28 elements, 65,536 segments (the headline):
    256 segments spread over the array (every launch-range boundary class is
    hit at this density), each against the oracle on its own slice;
  * u32 splitmix32 scan mod 2^32, 2^28: every output, bit for bit (the
    oracle's integer scan runs in a few seconds);
  * f32 compensated scan of x^2, 2^28: 4,096 sampled prefixes, each exact in
    the oracle and rounded once, within the given 1e-5 relative bar;
  * batched, 10,000 arrays: 200 sampled arrays against the oracle;
  * FP16 storage, Horner 8, 2^30: the whole sum, min and max (the oracle's
    exact sum over 2^26-element chunks, combined in FP64).
Inputs come from the same seeded generators as the benchmark."""
import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import map_error_bound, oracle_map, u32_host

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import binding, build
    build.build()
    binding.lib()
    return binding


def test_headline_segmented_sampled_segments(orc, B):
    x, m, off = I.rational_segments(1 << 28, 65536)
    n, nseg = x.size, off.size - 1
    xd = torch.from_numpy(x).cuda()
    offd = torch.from_numpy(off).cuda()
    sums = torch.empty(nseg, dtype=torch.float64, device="cuda")
    mins = torch.empty(nseg, dtype=torch.float32, device="cuda")
    maxs = torch.empty(nseg, dtype=torch.float32, device="cuda")
    ws = B.workspace(B.tr_segmented_reduce_workspace_size(n, nseg, B.TR_F32))
    ex = B.make_exec(ws)
    B.tr_segmented_reduce(m, xd, offd, B.TR_SUM | B.TR_MIN | B.TR_MAX, sums, mins, maxs, ex)
    B.tr_check(ex)
    s, lo, hi = sums.cpu().numpy(), mins.cpu().numpy().astype(np.float64), maxs.cpu().numpy().astype(np.float64)
    del xd
    spec = oracle_map(orc, m)
    pick = np.unique(np.concatenate([np.linspace(0, nseg - 1, 250).astype(np.int64), [0, 1, nseg - 2, nseg - 1]]))
    for k in pick:
        a, b = int(off[k]), int(off[k + 1])
        xs = x[a:b].astype(np.float64)
        rs, rlo, rhi = orc.reduce_float(spec, xs)
        f = orc.map_values(spec, xs)
        bnd = map_error_bound(m, xs, f)
        tol = 1e-6 * np.sum(np.abs(f)) + np.sum(bnd) + 1e-30
        assert abs(s[k] - rs) <= tol, (k, s[k], rs, tol)
        mb = np.max(bnd) + 2.0 ** -24 * max(abs(rlo), abs(rhi))
        assert abs(lo[k] - rlo) <= mb and abs(hi[k] - rhi) <= mb, k


def test_u32_scan_full_size_bitexact(orc, B):
    x = I.mixer_u32(1 << 28, stream="mixer_u32_scan")
    xd = torch.from_numpy(x.view(np.int32)).cuda()
    y = torch.empty_like(xd)
    ws = B.workspace(B.tr_scan_workspace_size(x.size, B.TR_U32, B.TR_U32))
    ex = B.make_exec(ws)
    B.tr_scan({"kind": "splitmix32"}, xd, y, ex)
    B.tr_check(ex)
    got = u32_host(y)
    del xd, y
    ref = orc.scan_u32(orc.MapSpec("splitmix32"), x)
    assert np.array_equal(got, ref)


def test_f32_scan_full_size_sampled_prefixes(orc, B):
    x = I.square_f32(1 << 28)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty_like(xd)
    ws = B.workspace(B.tr_scan_workspace_size(x.size, B.TR_F32, B.TR_F32))
    ex = B.make_exec(ws)
    B.tr_scan(I.simple_map("square"), xd, y, ex)
    B.tr_check(ex)
    pos = np.unique(np.concatenate([np.random.default_rng(5).integers(0, x.size, 4090),
                                    [0, 1, 8191, 8192, x.size - 1]]))
    got = y[torch.from_numpy(pos).cuda()].cpu().numpy().astype(np.float64)
    del xd, y
    ref = orc.scan_float_sampled(orc.MapSpec("square"), x, pos)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-30), np.max(np.abs(got - ref) / np.abs(ref))


def test_batched_full_config_sampled_arrays(orc, B):
    xs, lens, maps = I.batched(10000)
    dev = [torch.from_numpy(a).cuda() for a in xs]
    n = len(xs)
    sums = torch.zeros(n, dtype=torch.float64, device="cuda")
    mins = torch.zeros(n, dtype=torch.float32, device="cuda")
    maxs = torch.zeros(n, dtype=torch.float32, device="cuda")
    plan = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=False)
    plan.run()
    torch.cuda.synchronize()
    s, lo, hi = sums.cpu().numpy(), mins.cpu().numpy(), maxs.cpu().numpy()
    plan.close()
    del dev
    for a in np.random.default_rng(9).choice(n, 200, replace=False):
        xd64 = xs[a].astype(np.float64)
        spec = oracle_map(orc, maps[a])
        rs, rlo, rhi = orc.reduce_float(spec, xd64)
        f = orc.map_values(spec, xd64)
        bnd = map_error_bound(maps[a], xd64, f)
        assert abs(s[a] - rs) <= 1e-6 * np.sum(np.abs(f)) + np.sum(bnd) + 1e-30, (a, s[a], rs)
        mb = np.max(bnd) + 2.0 ** -24 * max(abs(rlo), abs(rhi))
        assert abs(lo[a] - rlo) <= mb and abs(hi[a] - rhi) <= mb, a


def test_f16_storage_full_size(orc, B):
    x, m = I.horner_f16(1 << 30)
    xd = torch.from_numpy(x.view(np.int16)).cuda().view(torch.float16)
    out = torch.empty(3, dtype=torch.float64, device="cuda")
    mm = torch.empty(2, dtype=torch.float32, device="cuda")
    ws = B.workspace(B.tr_reduce_workspace_size(x.size, B.TR_F16))
    ex = B.make_exec(ws)
    B.tr_reduce(m, xd, B.TR_SUM | B.TR_MIN | B.TR_MAX, out[0:1], mm[0:1], mm[1:2], ex)
    B.tr_check(ex)
    s, lo, hi = float(out[0]), float(mm[0]), float(mm[1])
    del xd
    spec = oracle_map(orc, m)
    total, sabs, bsum, rlo, rhi, bmax = 0.0, 0.0, 0.0, np.inf, -np.inf, 0.0
    step = 1 << 26
    for a in range(0, x.size, step):
        xc = x[a:a + step].astype(np.float64)
        rs, clo, chi = orc.reduce_float(spec, xc)
        f = orc.map_values(spec, xc)
        bnd = map_error_bound(m, xc, f)
        total += rs
        sabs += float(np.sum(np.abs(f)))
        bsum += float(np.sum(bnd))
        bmax = max(bmax, float(np.max(bnd)))
        rlo, rhi = min(rlo, clo), max(rhi, chi)
    assert abs(s - total) <= 1e-6 * sabs + bsum, (s, total)
    mb = bmax + 2.0 ** -24 * max(abs(rlo), abs(rhi))
    assert abs(lo - rlo) <= mb and abs(hi - rhi) <= mb
