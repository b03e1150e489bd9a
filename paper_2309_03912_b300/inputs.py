"""Seeded synthetic inputs for the transform-reduce-scan workloads.

This module is the only code shared by the CUDA path's callers and the oracle's
callers.  It holds no arithmetic of the method (no map evaluation, no sums, no
scans): it only draws random inputs with numpy's PCG64 and lays out their
structure (segment offsets, array lengths, map descriptors as plain data).

Every float input is drawn in FP64 and then rounded (nearest-even) to its
storage type; the rounded values are the inputs both sides see.  Coefficients
of maps evaluated in FP32 on the device are likewise rounded to FP32 here, so
that both sides use identical coefficient values.

Workloads (sizes are parameters; the defaults are the full benchmark sizes):

* ``horner_f64``   -- x ~ U[-1,1] f64, degree-8 Horner with N(0,1) coefficients.
* ``mixer_u32``    -- x uniform u32 (xorshift32 / splitmix32 inputs).
* ``rational_segments`` -- x ~ N(0,1) f32, rational P/Q of degree 6/6 whose Q
  has only even powers with positive coefficients (Q >= 1, no poles), and
  segment offsets with lengths ~ U{1..8192} rescaled to sum exactly to n.
* ``square_f32``   -- x ~ U[0,1] f32 (f(x) = x^2 scan).
* ``batched``      -- many f32 arrays with log-uniform lengths and a map drawn
  per array from {Horner deg 4-16, rational 6/6, 6-step Newton cube root}.
* ``vandermonde``  -- points x ~ U[-1,1] f32 and a (deg+1) x npoly coefficient
  matrix with C[k, j] ~ N(0,1)/(k+1) rounded to f32.
* ``horner_f16``   -- x ~ U[-1,1] rounded to f16, degree-8 Horner in FP32.
"""
from __future__ import annotations

import numpy as np

ROOT_SEED = 20230907
# one child stream per workload, fixed order (never reorder: it changes inputs)
_STREAMS = ["horner_f64", "mixer_u32", "rational_segments", "mixer_u32_scan", "square_f32",
            "batched", "vandermonde", "horner_f16", "misc"]

CHUNK = 1 << 24


def rng(stream: str, salt: int = 0) -> np.random.Generator:
    """PCG64 generator for a named workload stream (and an optional salt)."""
    ss = np.random.SeedSequence(ROOT_SEED)
    child = ss.spawn(len(_STREAMS))[_STREAMS.index(stream)]
    if salt:
        child = np.random.SeedSequence(entropy=child.entropy, spawn_key=child.spawn_key + (salt,))
    return np.random.Generator(np.random.PCG64(child))


def _chunked(g: np.random.Generator, n: int, dtype, draw) -> np.ndarray:
    """Draw n values in FP64 chunk by chunk (same stream as one call) and round."""
    out = np.empty(n, dtype=dtype)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        out[s:e] = draw(g, e - s).astype(dtype)
    return out


def uniform(g, n, lo, hi, dtype):
    return _chunked(g, n, dtype, lambda gg, k: gg.uniform(lo, hi, k))


def normal(g, n, dtype):
    return _chunked(g, n, dtype, lambda gg, k: gg.standard_normal(k))


def u32(g, n):
    out = np.empty(n, dtype=np.uint32)
    for s in range(0, n, CHUNK):
        e = min(n, s + CHUNK)
        out[s:e] = g.integers(0, 1 << 32, e - s, dtype=np.uint64).astype(np.uint32)
    return out


def f32_exact(v) -> np.ndarray:
    """FP64 array whose values are exactly representable in FP32."""
    return np.asarray(v, dtype=np.float64).astype(np.float32).astype(np.float64)


# --------------------------------------------------------------------------
# map descriptors as plain data: {"kind": str, "cp": list, "cq": list, "iters": int}
# --------------------------------------------------------------------------

def horner_map(coef) -> dict:
    return {"kind": "horner", "cp": [float(c) for c in coef], "cq": [1.0], "iters": 0}


def rational_map(cp, cq) -> dict:
    return {"kind": "rational", "cp": [float(c) for c in cp], "cq": [float(c) for c in cq], "iters": 0}


def newton_map(iters: int = 6) -> dict:
    return {"kind": "newton_cbrt", "cp": [0.0], "cq": [1.0], "iters": int(iters)}


def simple_map(kind: str) -> dict:
    return {"kind": kind, "cp": [0.0], "cq": [1.0], "iters": 0}


def positive_even_q(g: np.random.Generator, deg: int = 6) -> np.ndarray:
    """Q(x) = 1 + a_1 x^2 + a_2 x^4 + ... with a_k = |N(0,1)| + 0.1, so Q >= 1
    on the real line (no poles); odd coefficients are zero."""
    q = np.zeros(deg + 1)
    q[0] = 1.0
    for k in range(2, deg + 1, 2):
        q[k] = abs(g.standard_normal()) + 0.1
    return q


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------

def horner_f64(n: int = 1 << 20, deg: int = 8, salt: int = 0):
    g = rng("horner_f64", salt)
    coef = g.standard_normal(deg + 1)
    x = uniform(g, n, -1.0, 1.0, np.float64)
    return x, horner_map(coef)


def mixer_u32(n: int = 1 << 20, salt: int = 0, stream: str = "mixer_u32"):
    return u32(rng(stream, salt), n)


def segment_offsets(g: np.random.Generator, n: int, nseg: int, max_len: int = 8192) -> np.ndarray:
    """Offsets o_0 = 0 < ... <= o_nseg = n: lengths L_s ~ U{1..max_len}, rescaled
    by o_s = floor(n * P_s / P_nseg) (P = prefix sums of L, exact integers), then
    clamped so every segment is non-empty (when n >= nseg) and the total is n."""
    L = g.integers(1, max_len + 1, nseg, dtype=np.int64)
    P = np.concatenate([[0], np.cumsum(L)])
    S = int(P[-1])
    if S * max(n, 1) < (1 << 62):
        o = (P * n) // S
    else:  # exact big-integer arithmetic
        o = ((P.astype(object) * n) // S).astype(np.int64)
    o[0] = 0
    o[-1] = n
    if n >= nseg:
        for s in range(1, nseg + 1):          # forward: lengths >= 1
            if o[s] < o[s - 1] + 1:
                o[s] = o[s - 1] + 1
        for s in range(nseg - 1, 0, -1):      # backward: room for the rest
            lim = n - (nseg - s)
            if o[s] > lim:
                o[s] = lim
        o[-1] = n
    return o


def rational_segments(n: int = 1 << 28, nseg: int = 65536, salt: int = 0):
    g = rng("rational_segments", salt)
    cp = f32_exact(g.standard_normal(7))
    cq = f32_exact(positive_even_q(g, 6))
    offsets = segment_offsets(g, n, nseg)
    x = normal(g, n, np.float32)
    return x, rational_map(cp, cq), offsets


def square_f32(n: int = 1 << 28, salt: int = 0):
    g = rng("square_f32", salt)
    return uniform(g, n, 0.0, 1.0, np.float32)


def batched_lengths(g: np.random.Generator, n_arrays: int, log2_max: int = 20) -> np.ndarray:
    """L = min(2^log2_max, max(1, floor(2^(log2_max * u)))), u ~ U[0,1)."""
    u = g.random(n_arrays)
    L = np.floor(np.exp2(log2_max * u)).astype(np.int64)
    return np.clip(L, 1, 1 << log2_max)


def batched_maps(g: np.random.Generator, n_arrays: int) -> list:
    """Per array: kind uniform over {Horner, rational, Newton}; Horner degree
    ~ U{4..16} with N(0,1) coefficients; rational 6/6 with even positive Q."""
    maps = []
    kinds = g.integers(0, 3, n_arrays)
    for k in kinds:
        if k == 0:
            d = int(g.integers(4, 17))
            maps.append(horner_map(f32_exact(g.standard_normal(d + 1))))
        elif k == 1:
            maps.append(rational_map(f32_exact(g.standard_normal(7)), f32_exact(positive_even_q(g, 6))))
        else:
            maps.append(newton_map(6))
    return maps


def batched(n_arrays: int = 10000, log2_max: int = 20, salt: int = 0, with_data: bool = True):
    g = rng("batched", salt)
    lens = batched_lengths(g, n_arrays, log2_max)
    maps = batched_maps(g, n_arrays)
    xs = [uniform(g, int(L), -2.0, 2.0, np.float32) for L in lens] if with_data else None
    return xs, lens, maps


def vandermonde(m: int = 1 << 20, npoly: int = 4096, deg: int = 31, salt: int = 0):
    g = rng("vandermonde", salt)
    coef = f32_exact(g.standard_normal((deg + 1, npoly)) / (np.arange(deg + 1)[:, None] + 1.0))
    x = uniform(g, m, -1.0, 1.0, np.float32)
    return x, coef.astype(np.float32)


def horner_f16(n: int = 1 << 30, deg: int = 8, salt: int = 0):
    g = rng("horner_f16", salt)
    coef = f32_exact(g.standard_normal(deg + 1))
    x = uniform(g, n, -1.0, 1.0, np.float16)
    return x, horner_map(coef)
