"""hdc: the same map functions evaluated at compile time, on the host and on
the device must agree (the paper's thesis: one definition for all execution
spaces, Sec. 2.3 and Sec. 2.6, with the hdc trait of Sec. 4).

CPU part: g++ compiles tests/hdc_host_check.cpp against the product header
maps.h (compile time: its static_asserts; host: its evaluations), and the host
results are compared with the oracle -- bit for bit in FP64 (same fma and
division sequence) and for the integer mixers, within the derived FP32 error
bound in FP32.  The GPU part (test_gpu_parity.py) compares tr_map with the
same host build bit for bit.
"""
import os
import subprocess
import tempfile

import numpy as np
import pytest

from tests.helpers import map_error_bound, oracle_map

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2309_03912_b300", "csrc")


def build_host_check() -> str:
    out = os.path.join(tempfile.mkdtemp(), "hdc_host_check")
    subprocess.check_call(["g++", "-std=c++17", "-O2", "-ffp-contract=off", "-pthread", "-I" + CSRC,
                           os.path.join(ROOT, "tests", "hdc_host_check.cpp"), "-o", out])
    return out


@pytest.fixture(scope="module")
def host_bin():
    return build_host_check()


def host_eval(host_bin, m: dict, x, prec: str):
    d = tempfile.mkdtemp()
    fi, fo = os.path.join(d, "in.bin"), os.path.join(d, "out.bin")
    np.asarray(x, dtype=np.float64).tofile(fi)
    cp = [repr(float(c)) for c in m.get("cp", [0.0])]
    cq = [repr(float(c)) for c in m.get("cq", [1.0])]
    args = [host_bin, m["kind"], prec, fi, fo, str(m.get("iters", 6)), str(len(cp)), *cp, str(len(cq)), *cq]
    subprocess.check_call(args)
    return np.fromfile(fo, dtype=np.float64)


MAPS = [
    {"kind": "identity"},
    {"kind": "square"},
    {"kind": "horner", "cp": [0.5, -1.25, 2.0, 0.75, -0.3, 1.5, -2.25, 0.125, 1.0]},
    {"kind": "horner", "cp": list(np.random.default_rng(1).standard_normal(32).astype(np.float32).astype(float))},
    {"kind": "rational", "cp": [1.0, -0.5, 0.25, 2.0, -1.0, 0.5, 0.125], "cq": [1.0, 0, 0.7, 0, 0.3, 0, 0.2]},
    {"kind": "newton_cbrt", "iters": 6},
]


@pytest.mark.parametrize("m", MAPS, ids=lambda m: m["kind"])
def test_host_fp64_equals_oracle_bitwise(orc, host_bin, m):
    x = np.random.default_rng(2).uniform(-2, 2, 3000)
    x[:4] = [0.0, -0.0, 1.0, -1.0]
    y = host_eval(host_bin, m, x, "d")
    ref = orc.map_values(oracle_map(orc, m), x)
    assert np.array_equal(y.view(np.int64), ref.view(np.int64))


@pytest.mark.parametrize("m", MAPS, ids=lambda m: m["kind"])
def test_host_fp32_within_bound(orc, host_bin, m):
    x = np.random.default_rng(3).uniform(-2, 2, 3000).astype(np.float32).astype(np.float64)
    m32 = dict(m)
    for key in ("cp", "cq"):
        if key in m32:
            m32[key] = list(np.asarray(m32[key], dtype=np.float32).astype(float))
    y = host_eval(host_bin, m32, x, "f")
    ref = orc.map_values(oracle_map(orc, m32), x)
    assert np.all(np.abs(y - ref) <= map_error_bound(m32, x, ref))


@pytest.mark.parametrize("kind", ["xorshift32", "splitmix32"])
def test_host_mixers_equal_oracle(orc, host_bin, kind):
    x = np.random.default_rng(4).integers(0, 1 << 32, 5000, dtype=np.uint64).astype(np.uint32)
    y = host_eval(host_bin, {"kind": kind}, x.astype(np.float64), "d").astype(np.uint64).astype(np.uint32)
    assert np.array_equal(y, orc.map_values(orc.MapSpec(kind), x))


def test_div3_is_the_ieee_quotient_for_every_float(host_bin):
    """The division-free s / 3 of the FP32 Newton map (Markstein correction
    after a multiply by RN(1/3)) equals the IEEE quotient s / 3.0f bit for
    bit over all 2^32 inputs, subnormals, infinities and zeros included."""
    r = subprocess.run([host_bin, "div3"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and r.stdout.strip() == "0", (r.returncode, r.stdout, r.stderr)
