"""CPU oracle for the transform-reduce-scan path -- TEST INFRASTRUCTURE ONLY.

Only the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
leg of ``bench.py`` may import this package.  The product library never links,
calls or includes anything here, and nothing here imports the product package.

The arithmetic lives in ``tr_oracle.c`` (plain C loops, FP64 with explicit
``fma`` and exact fixed-point summation, exact integers); this module only
compiles it with gcc and marshals numpy arrays.  Each function cites the
definition it follows.

The paper (Mejstrik, "__host__ __device__ -- Generic programming in Cuda")
is about authoring such functions once for host, device and compile time; it
prescribes none of the arithmetic, so the definitions follow the textbook
methods named in ``tr_oracle.c``:

* Horner's rule with explicit fma; rational P/Q with one IEEE division;
  fixed-step Newton iterate for the cube root (the iterate, not cbrt);
* xorshift32 (Marsaglia 2003, shifts 13/17/5) and a splitmix-style 32-bit
  finaliser (constants from the golden ratio, sqrt 2 and sqrt 3);
* exact sums (Kulisch & Miranker fixed-point register) rounded once;
* inclusive scans whose every prefix is exact and rounded once.

Parity pins for every function live in ``tests/test_oracle_pins.py``; none of
them is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tr_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

# map kinds, by name (the oracle's own numbering, private to tr_oracle.c)
KINDS = {
    "identity": 0,
    "square": 1,
    "horner": 2,
    "rational": 3,
    "newton_cbrt": 4,
    "xorshift32": 5,
    "splitmix32": 6,
}


class _Map(ctypes.Structure):
    _fields_ = [
        ("kind", ctypes.c_int32),
        ("deg_p", ctypes.c_int32),
        ("deg_q", ctypes.c_int32),
        ("iters", ctypes.c_int32),
        ("cp", ctypes.c_void_p),
        ("cq", ctypes.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile tr_oracle.c into liboracle.so next to it (gcc, no fp contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared", "-pthread",
             _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P, I64, I32, U64 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_uint64
            lib.orc_exact_sum.argtypes = [P, I64, ctypes.c_int]
            lib.orc_exact_sum.restype = ctypes.c_double
            lib.orc_map_f64.argtypes = [P, P, P, I64]
            lib.orc_map_u32.argtypes = [I32, P, P, I64]
            lib.orc_reduce_f64.argtypes = [P, P, I64, P]
            lib.orc_reduce_u32.argtypes = [I32, P, I64, P, P, P]
            lib.orc_segreduce_f64.argtypes = [P, P, P, I64, P, P, P]
            lib.orc_mixer_range_sum.argtypes = [I32, U64, U64]
            lib.orc_mixer_range_sum.restype = U64
            lib.orc_scan_u32.argtypes = [I32, P, P, I64]
            lib.orc_scan_u32_u64.argtypes = [I32, P, P, I64]
            lib.orc_scan_f64.argtypes = [P, P, P, I64, ctypes.c_int]
            lib.orc_scan_f64_sampled.argtypes = [P, P, I64, P, I64, P, ctypes.c_int]
            lib.orc_vandermonde.argtypes = [P, P, I32, I64, P, I64, P, P]
            lib.orc_widen_f16.argtypes = [P, P, I64]
            lib.orc_scan_u32_excl.argtypes = [I32, P, P, I64]
            lib.orc_scan_u32_u64_excl.argtypes = [I32, P, P, I64]
            lib.orc_scan_f64_excl.argtypes = [P, P, P, I64, ctypes.c_int]
            lib.orc_reduce_mt.argtypes = [P, I32, P, I32, I64, P, I32]
            lib.orc_segreduce_mt.argtypes = [P, I32, P, I32, P, I64, P, P, P, P, I32]
            lib.orc_map_f32.argtypes = [P, P, P, I64]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


class MapSpec:
    """A map of the family, by name, with FP64 coefficients (ascending powers)."""

    def __init__(self, kind: str, cp=None, cq=None, iters: int = 6):
        self.kind = kind
        self.cp = np.ascontiguousarray(cp if cp is not None else [0.0], dtype=np.float64)
        self.cq = np.ascontiguousarray(cq if cq is not None else [1.0], dtype=np.float64)
        self.iters = int(iters)

    def _c(self) -> _Map:
        return _Map(KINDS[self.kind], len(self.cp) - 1, len(self.cq) - 1, self.iters,
                    _ptr(self.cp), _ptr(self.cq))


def _f64(x) -> np.ndarray:
    """Inputs of any float storage type are widened exactly to FP64."""
    return np.ascontiguousarray(np.asarray(x).astype(np.float64))


def _u32(x) -> np.ndarray:
    return np.ascontiguousarray(x, dtype=np.uint32)


def exact_sum(v, p: int = 53) -> float:
    """Exact sum of doubles, rounded once to nearest-even with p bits (53 or 24)."""
    v = _f64(v)
    return float(_load().orc_exact_sum(_ptr(v), v.size, int(p)))


def map_values(m: MapSpec, x) -> np.ndarray:
    """y_i = f(x_i): FP64 for float maps, u32 for the integer mixers."""
    lib = _load()
    if m.kind in ("xorshift32", "splitmix32") or (m.kind == "identity" and np.asarray(x).dtype == np.uint32):
        xu = _u32(x)
        y = np.empty_like(xu)
        lib.orc_map_u32(KINDS[m.kind], _ptr(xu), _ptr(y), xu.size)
        return y
    xd = _f64(x)
    y = np.empty_like(xd)
    c = m._c()
    lib.orc_map_f64(ctypes.byref(c), _ptr(xd), _ptr(y), xd.size)
    return y


def reduce_float(m: MapSpec, x):
    """(exact sum rounded to double, min, max) of f over x."""
    xd = _f64(x)
    out = np.empty(3, np.float64)
    c = m._c()
    _load().orc_reduce_f64(ctypes.byref(c), _ptr(xd), xd.size, _ptr(out))
    return float(out[0]), float(out[1]), float(out[2])


def reduce_u32(m: MapSpec, x):
    """(exact u64 sum, min, max) of the integer map over u32 input."""
    xu = _u32(x)
    s = np.zeros(1, np.uint64)
    lo = np.zeros(1, np.uint32)
    hi = np.zeros(1, np.uint32)
    _load().orc_reduce_u32(KINDS[m.kind], _ptr(xu), xu.size, _ptr(s), _ptr(lo), _ptr(hi))
    return int(s[0]), int(lo[0]), int(hi[0])


def segmented_reduce_float(m: MapSpec, x, offsets):
    """Per segment [off[s], off[s+1]): exact sum (double), min, max of f."""
    xd = _f64(x)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    sums = np.empty(nseg, np.float64)
    mins = np.empty(nseg, np.float64)
    maxs = np.empty(nseg, np.float64)
    c = m._c()
    _load().orc_segreduce_f64(ctypes.byref(c), _ptr(xd), _ptr(off), nseg, _ptr(sums), _ptr(mins), _ptr(maxs))
    return sums, mins, maxs


def mixer_range_sum(kind: str, lo: int, hi: int) -> int:
    """Exact sum of the mixer over the integers [lo, hi), hi <= 2^32."""
    return int(_load().orc_mixer_range_sum(KINDS[kind], lo, hi))


def scan_u32(m: MapSpec, x, exclusive: bool = False) -> np.ndarray:
    """Inclusive (or exclusive) scan of the integer map modulo 2^32."""
    xu = _u32(x)
    y = np.empty_like(xu)
    fn = _load().orc_scan_u32_excl if exclusive else _load().orc_scan_u32
    fn(KINDS[m.kind], _ptr(xu), _ptr(y), xu.size)
    return y


def scan_u32_u64(m: MapSpec, x, exclusive: bool = False) -> np.ndarray:
    """Inclusive (or exclusive) scan of the integer map widened to u64 (exact)."""
    xu = _u32(x)
    y = np.empty(xu.size, np.uint64)
    fn = _load().orc_scan_u32_u64_excl if exclusive else _load().orc_scan_u32_u64
    fn(KINDS[m.kind], _ptr(xu), _ptr(y), xu.size)
    return y


def scan_float(m: MapSpec, x, p: int = 24, exclusive: bool = False) -> np.ndarray:
    """Inclusive (or exclusive) scan: every prefix exact, rounded once to p bits (24: float)."""
    xd = _f64(x)
    y = np.empty_like(xd)
    c = m._c()
    fn = _load().orc_scan_f64_excl if exclusive else _load().orc_scan_f64
    fn(ctypes.byref(c), _ptr(xd), _ptr(y), xd.size, int(p))
    return y


def scan_float_sampled(m: MapSpec, x, positions, p: int = 24) -> np.ndarray:
    """Exact inclusive prefixes of f at the given positions, each rounded once."""
    xd = _f64(x)
    pos = np.ascontiguousarray(np.sort(np.asarray(positions, dtype=np.int64)))
    out = np.empty(pos.size, np.float64)
    c = m._c()
    _load().orc_scan_f64_sampled(ctypes.byref(c), _ptr(xd), xd.size, _ptr(pos), pos.size, _ptr(out), int(p))
    return out


def vandermonde(x, coef, rows=None, with_scale: bool = True):
    """Y[r, j] = sum_k coef[k, j] x[rows[r]]^k by FP64 Horner, and the scale
    S[r, j] = sum_k |coef[k, j]| |x|^k.  coef is (deg+1) x npoly."""
    xd = _f64(x)
    cd = np.ascontiguousarray(coef, dtype=np.float64)
    deg = cd.shape[0] - 1
    npoly = cd.shape[1]
    rr = np.arange(xd.size, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
    y = np.empty((rr.size, npoly), np.float64)
    s = np.empty((rr.size, npoly), np.float64) if with_scale else None
    _load().orc_vandermonde(_ptr(xd), _ptr(cd), deg, npoly, _ptr(rr), rr.size, _ptr(y),
                            _ptr(s) if s is not None else None)
    return (y, s) if with_scale else y


# ---------------------------------------------------------------------------- multi-threaded drivers

_IN = {np.dtype(np.float64): 0, np.dtype(np.float32): 1, np.dtype(np.float16): 2}


def host_threads() -> int:
    """Host cores this process may run on (its CPU affinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _stored(x) -> np.ndarray:
    """float16 / float32 / float64 arrays are passed as stored (widened exactly in C)."""
    a = np.asarray(x)
    if a.dtype not in _IN:
        a = a.astype(np.float64)
    return np.ascontiguousarray(a)


def widen_f16(h) -> np.ndarray:
    """Exact FP64 values of IEEE binary16 data (given as float16 or uint16 bits)."""
    hb = np.ascontiguousarray(np.asarray(h).view(np.uint16))
    y = np.empty(hb.size, np.float64)
    _load().orc_widen_f16(_ptr(hb), _ptr(y), hb.size)
    return y


def map_values_f32(m: MapSpec, x) -> np.ndarray:
    """y_i = f(x_i) evaluated in IEEE binary32 (the map's own operation sequence,
    one binary32 rounding per operation), widened to FP64.  Inputs and
    coefficients must be binary32 values."""
    xd = _f64(x)
    y = np.empty_like(xd)
    c = m._c()
    _load().orc_map_f32(ctypes.byref(c), _ptr(xd), _ptr(y), xd.size)
    return y


def reduce_float_mt(m: MapSpec, x, threads: int | None = None, f32: bool = False):
    """(exact sum, min, max, exact sum of |f|) of f over x (f16 / f32 / f64
    storage) on `threads` host threads; the same values for any thread count.
    f32: f evaluated in binary32 (map_values_f32) instead of FP64."""
    xs = _stored(x)
    out = np.empty(4, np.float64)
    c = m._c()
    _load().orc_reduce_mt(ctypes.byref(c), int(f32), _ptr(xs), _IN[xs.dtype], xs.size, _ptr(out),
                          int(threads or host_threads()))
    return float(out[0]), float(out[1]), float(out[2]), float(out[3])


def segmented_reduce_float_mt(m: MapSpec, x, offsets, threads: int | None = None, f32: bool = False):
    """segmented_reduce_float on `threads` host threads, plus the exact sum of
    |f| per segment: (sums, mins, maxs, abs_sums); f32 as for reduce_float_mt."""
    xs = _stored(x)
    off = np.ascontiguousarray(offsets, dtype=np.int64)
    nseg = off.size - 1
    sums, mins, maxs, abss = (np.empty(nseg, np.float64) for _ in range(4))
    c = m._c()
    _load().orc_segreduce_mt(ctypes.byref(c), int(f32), _ptr(xs), _IN[xs.dtype], _ptr(off), nseg, _ptr(sums),
                             _ptr(mins), _ptr(maxs), _ptr(abss), int(threads or host_threads()))
    return sums, mins, maxs, abss
