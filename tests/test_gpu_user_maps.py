"""User-supplied maps through the C++ entry points (include/tr.hpp).

tests/user_map_check.cu holds maps written the way the paper teaches
(functors tagged host-device for the Sec. 4 trait, a __host__ __device__
lambda wrapped by tr::hd_lambda as in Sec. 2.6) and instantiates the library's
kernel templates for them; its static_asserts check constant evaluation and
that an untagged functor is not accepted as a host-device map.  Here the
results are checked against the oracle:
  * a hand-written degree-8 Horner functor: device map == host evaluation of
    the same functor == the oracle's binary32 map, bit for bit; its reduction
    within 1e-6 normwise of the exact sum of those values, min / max exact;
  * a user rational functor on FP16 storage, segmented: sums within 1e-6
    normwise of the exact binary32-value sums, min / max exact;
  * the lambda fma(x, x, 1) (Horner [1, 0, 1]) scanned, inclusive and
    exclusive, with its fused sum / min / max.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from paper_2309_03912_b300 import inputs as I

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "user_map_check.cu")
OUT = os.path.join(ROOT, "_build", "libusermap.so")
P = ctypes.c_void_p


@pytest.fixture(scope="module")
def U():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import binding, build
    build.build()
    binding.lib()
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    pkg = os.path.dirname(build.LIB)
    cmd = ([build.NVCC] + build.FLAGS + ["--extended-lambda", "-shared", SRC, "-o", OUT, "-L" + pkg, "-ltr",
                                         "-Xlinker", "-rpath=" + pkg] + build.LINK)
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    L = ctypes.CDLL(OUT)
    L.user_horner8_host.argtypes = [P, P, P, ctypes.c_int64]
    L.user_horner8_map.argtypes = [P, P, P, ctypes.c_int64]
    L.user_horner8_reduce.argtypes = [P, P, ctypes.c_int64, P, P, P, P, ctypes.c_size_t]
    L.user_rational_segreduce_f16.argtypes = [P, ctypes.c_int, P, ctypes.c_int, P, ctypes.c_int64, P, ctypes.c_int64,
                                              P, P, P, P, ctypes.c_size_t]
    L.user_lambda_scan.argtypes = [P, P, ctypes.c_int64, ctypes.c_int, P, P, P, P, ctypes.c_size_t]
    return L, binding


def _ws(B, nbytes):
    return B.workspace(nbytes)


def test_horner8_functor(orc, U):
    L, B = U
    g = np.random.default_rng(81)
    c = I.f32_exact(g.standard_normal(9))
    n = 1_000_003
    x = g.uniform(-1.5, 1.5, n).astype(np.float32)
    cd = np.ascontiguousarray(c, np.float64)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    assert L.user_horner8_map(cd.ctypes.data, xd.data_ptr(), y.data_ptr(), n) == 0
    host = np.empty(n, np.float32)
    L.user_horner8_host(cd.ctypes.data, x.ctypes.data, host.ctypes.data, n)
    spec = orc.MapSpec("horner", c)
    f32 = orc.map_values_f32(spec, x)
    got = y.cpu().numpy()
    assert np.array_equal(got.view(np.int32), host.view(np.int32))
    assert np.array_equal(got.astype(np.float64), f32)
    ws = _ws(B, B.tr_reduce_workspace_size(n, B.TR_F32))
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    mm = torch.zeros(2, dtype=torch.float32, device="cuda")
    assert L.user_horner8_reduce(cd.ctypes.data, xd.data_ptr(), n, out.data_ptr(), mm.data_ptr(),
                                 mm.data_ptr() + 4, ws.data_ptr(), ws.numel()) == 0
    rs, rlo, rhi, ra = orc.reduce_float_mt(spec, x, f32=True)
    assert abs(float(out.item()) - rs) <= 1e-6 * ra
    assert float(mm[0].item()) == rlo and float(mm[1].item()) == rhi


def test_rational_functor_f16_segmented(orc, U):
    L, B = U
    g = np.random.default_rng(82)
    p = I.f32_exact(g.standard_normal(5))
    q = I.f32_exact(I.positive_even_q(g, 4))
    n = 2_000_017
    x = g.uniform(-2, 2, n).astype(np.float16)
    off = I.segment_offsets(g, n, 700, 8192)
    xd = torch.from_numpy(x.view(np.int16)).cuda().view(torch.float16)
    offd = torch.from_numpy(off).cuda()
    nseg = off.size - 1
    sums = torch.zeros(nseg, dtype=torch.float64, device="cuda")
    mins = torch.zeros(nseg, dtype=torch.float32, device="cuda")
    maxs = torch.zeros(nseg, dtype=torch.float32, device="cuda")
    ws = _ws(B, B.tr_segmented_reduce_workspace_size(n, nseg, B.TR_F16))
    pd, qd = np.ascontiguousarray(p, np.float64), np.ascontiguousarray(q, np.float64)
    assert L.user_rational_segreduce_f16(pd.ctypes.data, p.size - 1, qd.ctypes.data, q.size - 1, xd.data_ptr(), n,
                                         offd.data_ptr(), nseg, sums.data_ptr(), mins.data_ptr(), maxs.data_ptr(),
                                         ws.data_ptr(), ws.numel()) == 0
    spec = orc.MapSpec("rational", p, q)
    rs, rlo, rhi, ra = orc.segmented_reduce_float_mt(spec, x, off, f32=True)
    s = sums.cpu().numpy()
    assert np.all(np.abs(s - rs) <= 1e-6 * ra)
    ne = np.isfinite(rlo)
    assert np.array_equal(mins.cpu().numpy().astype(np.float64)[ne], rlo[ne])
    assert np.array_equal(maxs.cpu().numpy().astype(np.float64)[ne], rhi[ne])


@pytest.mark.parametrize("exclusive", [False, True], ids=["incl", "excl"])
def test_lambda_scan(orc, U, exclusive):
    L, B = U
    g = np.random.default_rng(83)
    n = 300_007
    x = g.uniform(-1, 1, n).astype(np.float32)
    xd = torch.from_numpy(x).cuda()
    y = torch.empty(n, dtype=torch.float32, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    mm = torch.zeros(2, dtype=torch.float32, device="cuda")
    ws = _ws(B, B.tr_scan_workspace_size(n, B.TR_F32, B.TR_F32))
    assert L.user_lambda_scan(xd.data_ptr(), y.data_ptr(), n, int(exclusive), out.data_ptr(), mm.data_ptr(),
                              mm.data_ptr() + 4, ws.data_ptr(), ws.numel()) == 0
    spec = orc.MapSpec("horner", [1.0, 0.0, 1.0])  # fma(fma(1, x, 0), x, 1) = fma(x, x, 1)
    ref = orc.scan_float(spec, x, 24, exclusive=exclusive)
    got = y.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(got - ref) <= 1e-5 * np.abs(ref) + 1e-38)  # all terms >= 1
    rs, rlo, rhi, ra = orc.reduce_float_mt(spec, x, f32=True)
    assert abs(float(out.item()) - rs) <= 1e-6 * ra
    assert float(mm[0].item()) == rlo and float(mm[1].item()) == rhi
