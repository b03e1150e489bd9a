"""Parity at the benchmark's full sizes, in the launch configurations the
benchmark times, against the oracle (run on all host cores):

  * segmented rational 6/6, 2^28 elements, 65,536 segments (the headline):
    every segment's sum within the stated bar of 1e-6 normwise
    (|s - s_ref| / sum |f_ref|), min and max within 1e-5 of max |f_ref|;
  * u32 splitmix32 scan mod 2^32, 2^28: every output, bit for bit;
  * f32 compensated scan of x^2, 2^28: 4,096 sampled prefixes, each exact in
    the oracle and rounded once, within the stated 1e-5 relative bar;
  * batched, 10,000 arrays: every array's compensated sum within 1e-6
    normwise of the exact sum of its binary32 map values (bit-identical to the
    device's), min and max equal to theirs; the error against FP64 evaluation,
    which includes the FP32 map's own rounding (up to ~2e-5 for degree-16
    Horner at |x| near 2), is printed;
  * FP16 storage, Horner 8, 2^30: the whole sum within 1e-6 normwise, min and
    max within 1e-5 of max |f_ref|.
The per-element error bounds derived from the FP32 arithmetic (tests/helpers)
are printed beside the achieved errors as a diagnostic.
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


def _minmax_err(lo, hi, rlo, rhi):
    lo, hi, rlo, rhi = (np.atleast_1d(np.asarray(v, dtype=np.float64)) for v in (lo, hi, rlo, rhi))
    scale = np.maximum(np.maximum(np.abs(rlo), np.abs(rhi)), 1e-300)
    return float(np.max(np.maximum(np.abs(lo - rlo), np.abs(hi - rhi)) / scale))


def test_headline_segmented_all_segments(orc, B):
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
    s, lo, hi = sums.cpu().numpy(), mins.cpu().numpy(), maxs.cpu().numpy()
    del xd
    spec = oracle_map(orc, m)
    rs, rlo, rhi, ra = orc.segmented_reduce_float_mt(spec, x, off)
    err = np.abs(s - rs) / ra
    assert err.max() <= 1e-6, (int(np.argmax(err)), err.max())
    emm = _minmax_err(lo, hi, rlo, rhi)
    assert emm <= 1e-5, emm
    # diagnostic: the derived per-element bound summed over the worst segment
    k = int(np.argmax(err))
    a, b = int(off[k]), int(off[k + 1])
    xs = x[a:b].astype(np.float64)
    bound = np.sum(map_error_bound(m, xs, orc.map_values(spec, xs))) / ra[k]
    print(f"headline: max normwise sum error {err.max():.3g} (segment {k}; derived bound there {bound:.3g}), "
          f"min/max {emm:.3g}")


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


def test_batched_full_config_all_arrays(orc, B):
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
    es, e64, em64 = np.zeros(n), np.zeros(n), np.zeros(n)
    for a in range(n):
        spec = oracle_map(orc, maps[a])
        th = None if xs[a].size >= 65536 else 1
        # the FP32 map values (bit-identical on the device): compensated sums within 1e-6 normwise,
        # min / max exact
        rs, rlo, rhi, ra = orc.reduce_float_mt(spec, xs[a], th, f32=True)
        es[a] = abs(s[a] - rs) / max(ra, 1e-300)
        assert lo[a] == rlo and hi[a] == rhi, a
        # against FP64 evaluation: the FP32 map's own error included (reported)
        rs, rlo, rhi, ra = orc.reduce_float_mt(spec, xs[a], th)
        e64[a] = abs(s[a] - rs) / max(ra, 1e-300)
        em64[a] = _minmax_err(lo[a], hi[a], rlo, rhi)
    assert es.max() <= 1e-6, (int(np.argmax(es)), es.max())
    print(f"batched: max normwise sum error {es.max():.3g} against the binary32 map values, "
          f"{e64.max():.3g} against FP64 evaluation (min/max {em64.max():.3g}) over {n} arrays")


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
    rs, rlo, rhi, ra = orc.reduce_float_mt(oracle_map(orc, m), x)
    err = abs(s - rs) / ra
    emm = _minmax_err(lo, hi, rlo, rhi)
    assert err <= 1e-6, err
    assert emm <= 1e-5, emm
    print(f"f16 storage: normwise sum error {err:.3g}, min/max {emm:.3g}")
