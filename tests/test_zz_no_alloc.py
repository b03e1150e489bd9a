"""tr_scan_noalloc: the scan for callers that cannot allocate device memory.

Callers such as code running inside a memory allocator, plugins that are
handed only input and output pointers, or loops that must not allocate once
started cannot supply a workspace; tr_scan_noalloc keeps its scratch in a
fixed array inside the library instead.  This test calls it through the C ABI
twice in a row (the second call finds the first call's leftovers in the shared
array) and checks each output against the oracle with the tolerances used by
the other scan tests: bit for bit for the integer scans (u32 -> u32 mod 2^32
and u32 -> u64), 1e-5 relative per output for the compensated f32 scan of
x^2 >= 0 (the oracle's prefixes are exact, rounded once).  It also checks that sizes beyond the array's
limit are rejected with a message naming the limit.

This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I
from tests.helpers import u32_host, u64_host

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

LIMIT = 1 << 26


@pytest.fixture(scope="module")
def B():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import binding, build
    build.build()
    binding.lib()
    return binding


def _noalloc_twice(B, m, x, y_dtype):
    outs = []
    for _ in range(2):
        y = torch.full((x.numel(),), -1, dtype=y_dtype, device="cuda")
        status = torch.full((1,), 99, dtype=torch.int32, device="cuda")
        B.tr_scan_noalloc(m, x, y, status=status)
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        outs.append(y)
    return outs


@pytest.mark.parametrize("n", [1, 4097, 3_000_001, LIMIT])
def test_u32_scans_match_the_oracle_bitwise(orc, B, n):
    xh = I.u32(I.rng("misc", 21), n)
    x = torch.from_numpy(xh.view(np.int32)).cuda()
    m = {"kind": "splitmix32"}
    spec = orc.MapSpec("splitmix32")
    for y_dtype, ref, host in ((torch.int32, orc.scan_u32(spec, xh), u32_host),
                               (torch.int64, orc.scan_u32_u64(spec, xh), u64_host)):
        for y in _noalloc_twice(B, m, x, y_dtype):
            assert np.array_equal(host(y), ref)


@pytest.mark.parametrize("n", [1_000_003, (1 << 25) + 12_345])
def test_f32_scan_matches_the_oracle_within_tolerance(orc, B, n):
    xh = np.random.default_rng(22).uniform(0, 1, n).astype(np.float32)
    x = torch.from_numpy(xh).cuda()
    ref = orc.scan_float(orc.MapSpec("square"), xh, 24)
    for y in _noalloc_twice(B, I.simple_map("square"), x, torch.float32):
        got = y.double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-38)


def test_rejects_sizes_beyond_the_limit(B):
    L = B.lib()
    md = B.MapDesc({"kind": "splitmix32"})
    st = L.tr_scan_noalloc(md.ref(), None, B.TR_U32, None, B.TR_U32, LIMIT + 1, None, None, None)
    assert st == 1
    msg = L.tr_last_error().decode()
    assert "limit" in msg and str(LIMIT) in msg
