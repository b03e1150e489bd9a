"""Test helpers: oracle map specs, tolerances derived from the arithmetic of
each FP32 map, and device tensor plumbing.

Error bounds (u = 2^-24, FP32 compute; inputs and coefficients are exact FP32
values, so only the evaluation rounds):
  * Horner, degree d:  |p_hat - p| <= gamma_{2d+1} * sum_k |c_k| |x|^k
    (Higham, Accuracy and Stability of Numerical Algorithms, Sec. 5.1);
  * rational P/Q:      |r_hat - r| <= (gamma_{2dp+1} S_P + |r| gamma_{2dq+1} S_Q) / |Q|
                                      + 2u |r|   (first order);
  * square:            u |x^2|;
  * Newton cube root:  each step perturbs y by a few u|y| and propagates the
    previous error with factor |2/3 - 2x / (3 y^3)|; the bound accumulates
    that along the FP64 iterate path;
  * identity: exact.
A sum of n mapped values then carries sum_i bound_i plus its own summation
error (compensated: ~2u sum |f|, bounded in the tests by 1e-6 sum |f|).
"""
from __future__ import annotations

import math

import numpy as np

U32 = 2.0 ** -24


def gamma(k: int, u: float = U32) -> float:
    return k * u / (1 - k * u)


def oracle_map(orc, m: dict):
    return orc.MapSpec(m["kind"], m.get("cp"), m.get("cq"), m.get("iters", 6))


def _horner_abs(c, x):
    c = np.abs(np.asarray(c, dtype=np.float64))
    ax = np.abs(x)
    p = np.full_like(ax, c[-1])
    for ck in c[-2::-1]:
        p = p * ax + ck
    return p


def _horner(c, x):
    c = np.asarray(c, dtype=np.float64)
    p = np.full_like(x, c[-1])
    for ck in c[-2::-1]:
        p = p * x + ck
    return p


def map_error_bound(m: dict, x: np.ndarray, ref: np.ndarray) -> np.ndarray:
    """Per-element absolute error bound of the FP32 evaluation of map m at x
    (x: FP64 values of the FP32/FP16/BF16 inputs; ref: FP64 oracle values)."""
    x = np.asarray(x, dtype=np.float64)
    k = m["kind"]
    if k == "identity":
        return np.zeros_like(x)
    if k == "square":
        return U32 * np.abs(ref)
    if k == "horner":
        d = len(m["cp"]) - 1
        return gamma(2 * d + 1) * _horner_abs(m["cp"], x) + 1e-45
    if k == "rational":
        dp, dq = len(m["cp"]) - 1, len(m["cq"]) - 1
        sp = _horner_abs(m["cp"], x)
        sq = _horner_abs(m["cq"], x)
        q = np.abs(_horner(m["cq"], x))
        return (gamma(2 * dp + 1) * sp + np.abs(ref) * gamma(2 * dq + 1) * sq) / q * 1.01 + 2 * U32 * np.abs(ref) + 1e-45
    if k == "newton_cbrt":
        it = int(m.get("iters", 6))
        y = np.where(np.signbit(x), -1.0, 1.0)
        err = np.zeros_like(x)
        for _ in range(it):
            amp = np.abs(2.0 / 3.0 - 2.0 * x / (3.0 * y ** 3))
            y_next = (2.0 * y + x / (y * y)) / 3.0
            err = amp * err + 6 * U32 * (np.abs(y_next) + np.abs(x / (y * y)) / 3 + 2 * np.abs(y) / 3)
            y = y_next
        return err * 1.5 + 1e-45
    raise ValueError(k)


def to_dev(a: np.ndarray, dtype=None, offset: int = 0):
    """Copy a numpy array to the GPU; offset > 0 returns a view starting
    `offset` elements into a larger buffer (a misaligned base pointer)."""
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a))
    if t.dtype == torch.uint32:
        t = t.view(torch.int32)
    if dtype is not None:
        t = t.to(dtype)
    if offset:
        buf = torch.empty(t.numel() + offset, dtype=t.dtype, device="cuda")
        view = buf[offset:]
        view.copy_(t.cuda())
        return view
    return t.cuda()


def u32_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def u64_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint64)


def fsum(v):
    return math.fsum(np.asarray(v, dtype=np.float64))
