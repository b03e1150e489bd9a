"""The division-free FP32 quotient of the maps equals the IEEE division.

The rational map P/Q and the Newton step x / y^2 divide on the device by a
hardware reciprocal refined once, a product and one remainder correction
(Markstein 1990), on operands whose magnitudes lie in [2^-62, 2^62); all
other operands take the IEEE division.  Bit-identity with the IEEE quotient
(and so with the host and constant evaluations of the same map, the paper's
point in Sec. 2.3 and 2.6) rests on three checks made here on the GPU:

  * the hardware reciprocal is sign- and scale-invariant over every normal
    input whose reciprocal is normal (all 2^32 bit patterns);
  * the packed quotient equals a / b, and the negated form the Newton map
    runs on its negated iterate equals -(a / b), for every pair of
    significands in [1, 2) x [1, 2) (all 2^46 pairs, about a minute on a
    B300);
  * on the fast domain every intermediate stays normal (or is an exactly
    representable remainder), so the sequence commutes with scaling a and b by
    powers of two and with their signs: the two exhaustive checks then cover
    the whole fast domain.

A random sample over all exponents, the guard's edges and the special values
(zeros, subnormals, infinities, NaN) checks the guard itself.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "div_check.cu")
OUT = os.path.join(ROOT, "_build", "libdivcheck.so")


class Report(ctypes.Structure):
    _fields_ = [("mismatches", ctypes.c_ulonglong), ("recorded", ctypes.c_uint), ("pad", ctypes.c_uint),
                ("a", ctypes.c_uint * 16), ("b", ctypes.c_uint * 16)]


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2309_03912_b300 import build as bd
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    cmd = [bd.NVCC] + bd.FLAGS + ["-shared", SRC, "-o", OUT]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(OUT)
    L.div_check_rcp_invariance.argtypes = [ctypes.POINTER(Report)]
    L.div_check_significands.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.POINTER(Report)]
    L.div_check_values.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.POINTER(Report)]
    torch.cuda.init()
    return L


def _show(r: Report) -> str:
    return ", ".join(f"a={r.a[k]:08x} b={r.b[k]:08x}" for k in range(min(r.recorded, 16)))


def test_rcp_sign_and_scale_invariant(lib):
    r = Report()
    assert lib.div_check_rcp_invariance(ctypes.byref(r)) == 0
    assert r.mismatches == 0, _show(r)


@pytest.mark.slow
def test_all_significand_pairs_exact(lib):
    r = Report()
    assert lib.div_check_significands(0, 1 << 23, ctypes.byref(r)) == 0
    assert r.mismatches == 0, _show(r)


def test_guard_and_special_values(lib):
    g = np.random.default_rng(2023)
    n = 1 << 24
    # magnitudes spread over every exponent, random signs and significands
    def spread(k):
        bits = g.integers(0, 1 << 31, k, dtype=np.uint32) | (g.integers(0, 2, k, dtype=np.uint32) << 31)
        return bits.view(np.float32)
    a, b = spread(n), spread(n)
    edges = np.array([2.0 ** -62, 2.0 ** 62, np.nextafter(np.float32(2.0 ** -62), np.float32(0)),
                      np.nextafter(np.float32(2.0 ** 62), np.float32(np.inf)), np.float32(2.0 ** -62) * 3,
                      1.0, -1.0, 0.0, -0.0, np.inf, -np.inf, np.nan, 1e-45, -1e-45, 1.17549435e-38,
                      3.4028235e38, -3.4028235e38, 2.0 - 2.0 ** -23, 1.5], dtype=np.float32)
    ea, eb = np.meshgrid(edges, edges)
    a = np.concatenate([a, ea.ravel(), g.uniform(-1e3, 1e3, 1 << 20).astype(np.float32)])
    b = np.concatenate([b, eb.ravel(), g.uniform(1.0, 1e3, 1 << 20).astype(np.float32)])
    ad, bd = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    r = Report()
    assert lib.div_check_values(ad.data_ptr(), bd.data_ptr(), a.size, ctypes.byref(r)) == 0
    assert r.mismatches == 0, _show(r)
