"""Batched reduction (tr_batched_*): many arrays of uneven length, mixed maps,
one persistent launch from a CUDA graph -- against the oracle per array,
against the unbatched baseline (one tr_reduce per array), and for bitwise
determinism across runs.  Tolerances as for tr_reduce: the sum within
1e-6 * sum|f| plus the summed per-element map error bounds; min / max within
the largest element bound."""
import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import map_error_bound, oracle_map

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


def _workload(n_arrays=300, log2_max=16):
    xs, lens, maps = I.batched(n_arrays, log2_max, salt=3)
    g = np.random.default_rng(31)
    extra = [  # forms outside the fixed-degree fast paths, and edge lengths
        (g.uniform(-2, 2, 70_000).astype(np.float32), I.horner_map(I.f32_exact(g.standard_normal(21)))),
        (g.uniform(-2, 2, 5).astype(np.float32), I.rational_map(I.f32_exact(g.standard_normal(4)),
                                                                  I.f32_exact(I.positive_even_q(g, 4)))),
        (g.uniform(-2, 2, 1).astype(np.float32), I.newton_map(3)),
        (g.uniform(-2, 2, 100_001).astype(np.float32), I.simple_map("square")),
        (np.zeros(0, np.float32), I.simple_map("identity")),
    ]
    xs = list(xs) + [e[0] for e in extra]
    maps = list(maps) + [e[1] for e in extra]
    return xs, maps


def _check(orc, xs, maps, sums, mins, maxs):
    s, lo, hi = sums.cpu().numpy(), mins.cpu().numpy(), maxs.cpu().numpy()
    for a, (x, m) in enumerate(zip(xs, maps)):
        xd = x.astype(np.float64)
        ref = orc.map_values(oracle_map(orc, m), xd)
        rs, rlo, rhi = orc.reduce_float(oracle_map(orc, m), xd)
        b = map_error_bound(m, xd, ref)
        tol = 1e-6 * np.sum(np.abs(ref)) + np.sum(b) + 1e-30
        assert abs(s[a] - rs) <= tol, (a, m["kind"], s[a], rs)
        if x.size:
            mb = np.max(b) + 2.0 ** -24 * max(abs(rlo), abs(rhi))
            assert abs(lo[a] - rlo) <= mb and abs(hi[a] - rhi) <= mb
        else:
            assert s[a] == 0 and np.isposinf(lo[a]) and np.isneginf(hi[a])


@pytest.fixture(scope="module")
def batch(B):
    xs, maps = _workload()
    dev = [torch.from_numpy(x).cuda() for x in xs]
    n = len(xs)
    sums = torch.zeros(n, dtype=torch.float64, device="cuda")
    mins = torch.zeros(n, dtype=torch.float32, device="cuda")
    maxs = torch.zeros(n, dtype=torch.float32, device="cuda")
    return xs, maps, dev, sums, mins, maxs


def test_batched_graph_matches_oracle_and_is_deterministic(orc, B, batch):
    xs, maps, dev, sums, mins, maxs = batch
    plan = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=False)
    assert "tile=" in plan.describe()
    plan.run()
    torch.cuda.synchronize()
    _check(orc, xs, maps, sums, mins, maxs)
    first = (sums.clone(), mins.clone(), maxs.clone())
    for _ in range(3):
        sums.zero_(), mins.zero_(), maxs.zero_()
        plan.run()
        torch.cuda.synchronize()
        assert torch.equal(sums, first[0]) and torch.equal(mins, first[1]) and torch.equal(maxs, first[2])
    plan.close()


@pytest.mark.parametrize("use_graph", [False, True])
def test_unbatched_baseline_agrees(orc, B, batch, use_graph):
    xs, maps, dev, sums, mins, maxs = batch
    plan = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=False)
    sums.zero_(), mins.zero_(), maxs.zero_()
    plan.run_unbatched(use_graph)
    plan.run_unbatched(use_graph)
    torch.cuda.synchronize()
    _check(orc, xs, maps, sums, mins, maxs)
    plan.close()


def test_autotuned_plan(orc, B, batch, tmp_path, monkeypatch):
    xs, maps, dev, sums, mins, maxs = batch
    monkeypatch.setenv("TR_AUTOTUNE_CACHE", str(tmp_path / "tune.tsv"))
    plan = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=True)
    assert "autotuned" in plan.describe()
    sums.zero_()
    plan.run()
    torch.cuda.synchronize()
    _check(orc, xs, maps, sums, mins, maxs)
    plan.close()
    plan2 = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=True)  # served from the cache
    assert "cache" in plan2.describe()
    plan2.close()


def test_plan_validation(B):
    x = torch.zeros(10, device="cuda")
    s = torch.zeros(1, dtype=torch.float64, device="cuda")
    with pytest.raises(B.TrError):
        B.BatchPlan([x], [{"kind": "xorshift32"}], s, None, None, ops=B.TR_SUM)
    with pytest.raises(B.TrError):
        B.BatchPlan([x], [I.simple_map("square")], None, None, None, ops=B.TR_SUM)


@pytest.mark.parametrize("dt", [torch.float16, torch.bfloat16], ids=["f16", "bf16"])
def test_batched_low_precision_storage(orc, B, dt):
    """FP16 / BF16 storage with FP32 compute: every array against the oracle's
    binary32 map values of the stored inputs (compensated sums within 1e-6
    normwise, min / max exact), and equal to the per-array launches of the
    same storage."""
    xs, maps = _workload(120, 15)
    dev = [torch.from_numpy(x).to(dt).cuda() for x in xs]
    n = len(xs)
    out = [torch.zeros(n, dtype=torch.float64, device="cuda")] + \
          [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    plan = B.BatchPlan(dev, maps, *out, autotune=False)
    plan.run()
    torch.cuda.synchronize()
    s, lo, hi = (t.cpu().numpy() for t in out)
    for a, (x, m) in enumerate(zip(dev, maps)):
        xv = x.cpu().double().numpy()
        rs, rlo, rhi, ra = orc.reduce_float_mt(oracle_map(orc, m), xv, 1, f32=True)
        assert abs(s[a] - rs) <= 1e-6 * ra + 1e-30, (a, m["kind"])
        if xv.size:
            assert lo[a] == rlo and hi[a] == rhi, a
    ref = [torch.zeros_like(t) for t in out]
    plan2 = B.BatchPlan(dev, maps, *ref, autotune=False)
    plan2.run_unbatched(False)
    torch.cuda.synchronize()
    assert torch.equal(out[1], ref[1]) and torch.equal(out[2], ref[2])  # min / max: same values
    s2 = ref[0].cpu().numpy()
    for a, (x, m) in enumerate(zip(dev, maps)):
        rs, _, _, ra = orc.reduce_float_mt(oracle_map(orc, m), x.cpu().double().numpy(), 1, f32=True)
        assert abs(s2[a] - rs) <= 1e-6 * ra + 1e-30, a
    plan.close()
    plan2.close()


@pytest.mark.parametrize("dt", [torch.float32, torch.float16], ids=["f32", "f16"])
@pytest.mark.parametrize("threads,vectors", [(128, 2), (256, 2), (128, 4), (256, 4)])
def test_every_launch_shape_matches_oracle(orc, B, dt, threads, vectors, tmp_path, monkeypatch):
    """Each block size and count of vectors in flight per lane (the kernel's
    two instantiations), forced through the autotune cache: every array
    against the oracle's binary32 map of its stored values (sums within 1e-6
    normwise, min / max exact)."""
    xs, maps = _workload(150, 15)
    dev = [torch.from_numpy(x).to(dt).cuda() for x in xs]
    n = len(xs)
    out = [torch.zeros(n, dtype=torch.float64, device="cuda")] + \
          [torch.zeros(n, dtype=torch.float32, device="cuda") for _ in range(2)]
    cache = tmp_path / "tune.tsv"
    monkeypatch.setenv("TR_AUTOTUNE_CACHE", str(cache))
    B.BatchPlan(dev, maps, *out, autotune=True).close()  # writes this workload's cache line
    key = cache.read_text().splitlines()[0].split("\t")[0]
    cache.write_text(f"{key}\t8192\t{threads}\t1\t{vectors}\n")
    plan = B.BatchPlan(dev, maps, *out, autotune=True)
    d = plan.describe()
    assert "cache" in d and f"threads={threads}" in d and f"vectors_per_lane={vectors}" in d, d
    for t in out:
        t.zero_()
    plan.run()
    torch.cuda.synchronize()
    s, lo, hi = (t.cpu().numpy() for t in out)
    for a, (x, m) in enumerate(zip(dev, maps)):
        xv = x.cpu().double().numpy()
        rs, rlo, rhi, ra = orc.reduce_float_mt(oracle_map(orc, m), xv, 1, f32=True)
        assert abs(s[a] - rs) <= 1e-6 * ra + 1e-30, (a, m["kind"])
        if xv.size:
            assert lo[a] == rlo and hi[a] == rhi, a
        else:
            assert s[a] == 0 and np.isposinf(lo[a]) and np.isneginf(hi[a])
    plan.close()


def test_cache_line_without_vectors_field_reads_as_four(B, batch, tmp_path, monkeypatch):
    """A cache line of the older four-field form (no vectors per lane) is still
    served, with four vectors per lane."""
    xs, maps, dev, sums, mins, maxs = batch
    cache = tmp_path / "tune.tsv"
    monkeypatch.setenv("TR_AUTOTUNE_CACHE", str(cache))
    B.BatchPlan(dev, maps, sums, mins, maxs, autotune=True).close()
    key = cache.read_text().splitlines()[0].split("\t")[0]
    cache.write_text(f"{key}\t16384\t128\t0\n")
    plan = B.BatchPlan(dev, maps, sums, mins, maxs, autotune=True)
    d = plan.describe()
    assert "cache" in d and "tile=16384" in d and "vectors_per_lane=4" in d, d
    plan.close()
