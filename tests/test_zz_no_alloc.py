"""tr_scan_noalloc: the scan for callers that cannot allocate device memory.

Callers such as code running inside a memory allocator, plugins that are
handed only input and output pointers, or loops that must not allocate once
started cannot supply a workspace; tr_scan_noalloc keeps its scratch in a
fixed array inside the library instead.  This test calls it through the C ABI
twice in a row (the second call finds the first call's leftovers in the shared
array) and checks its output against tr_scan's with the tolerances used by the
other scan tests: bit for bit for integer scans, 1e-5 relative for the
compensated f32 scan of x^2 >= 0.  It also checks that sizes beyond the array's
limit are rejected with a message naming the limit.

This file sorts last so that a run stopping at the first failure has run
every other test first; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I

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


def _ref_scan(B, m, x, y_dtype):
    n = x.numel()
    y = torch.empty(n, dtype=y_dtype, device="cuda")
    ws = B.workspace(B.tr_scan_workspace_size(n, B.dtype_of(x), B.dtype_of(y)))
    ex = B.make_exec(ws)
    B.tr_scan(m, x, y, ex)
    B.tr_check(ex)
    return y


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
def test_u32_scans_match_tr_scan_bitwise(B, n):
    x = torch.from_numpy(I.u32(I.rng("misc", 21), n).view(np.int32)).cuda()
    m = {"kind": "splitmix32"}
    for y_dtype in (torch.int32, torch.int64):
        ref = _ref_scan(B, m, x, y_dtype).cpu().numpy()
        for y in _noalloc_twice(B, m, x, y_dtype):
            assert np.array_equal(y.cpu().numpy(), ref)


def test_f32_scan_matches_tr_scan_within_tolerance(B):
    n = 1_000_003
    x = torch.from_numpy(np.random.default_rng(22).uniform(0, 1, n).astype(np.float32)).cuda()
    m = I.simple_map("square")
    ref = _ref_scan(B, m, x, torch.float32).double().cpu().numpy()
    for y in _noalloc_twice(B, m, x, torch.float32):
        got = y.double().cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-38)


def test_rejects_sizes_beyond_the_limit(B):
    L = B.lib()
    md = B.MapDesc({"kind": "splitmix32"})
    st = L.tr_scan_noalloc(md.ref(), None, B.TR_U32, None, B.TR_U32, LIMIT + 1, None, None, None)
    assert st == 1
    msg = L.tr_last_error().decode()
    assert "limit" in msg and str(LIMIT) in msg
