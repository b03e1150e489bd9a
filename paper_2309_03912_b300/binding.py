"""Python binding of libtr (ctypes): the C-ABI names, argument marshalling only.

Every ``tr_*`` function here forwards to the entry point of the same name in
``libtr.so`` (declared in ``include/tr.h``); torch tensors supply device
memory and ``torch.cuda.current_stream()`` the stream.  Nothing is computed
here, and there is no fallback: if the library is missing, ``lib()`` raises.

Tensor dtypes map to tr_dtype as float16 -> F16, bfloat16 -> BF16,
float32 -> F32, float64 -> F64, int32/uint32 -> U32 and int64/uint64 -> U64
(signed integer tensors are reinterpreted bit for bit as unsigned).

Maps are plain dicts ``{"kind": str, "cp": [...], "cq": [...], "iters": int}``
as produced by ``paper_2309_03912_b300.inputs``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtr.so")

TR_F16, TR_BF16, TR_F32, TR_F64, TR_U32, TR_U64, TR_NONE = 0, 1, 2, 3, 4, 5, 15
TR_SUM, TR_MIN, TR_MAX = 1, 2, 4
TR_PREC_BF16X3, TR_PREC_FP32, TR_PREC_BF16X6 = 0, 1, 2
MAP_KINDS = {"identity": 0, "square": 1, "horner": 2, "rational": 3, "newton_cbrt": 4,
             "xorshift32": 5, "splitmix32": 6}
STATUS = {0: "TR_OK", 1: "TR_ERR_INVALID_ARG", 2: "TR_ERR_ALIGNMENT", 3: "TR_ERR_UNSUPPORTED",
          4: "TR_ERR_WORKSPACE", 5: "TR_ERR_CUDA", 6: "TR_ERR_TIMEOUT", 7: "TR_ERR_DEVICE_ASSERT"}

_DT = {torch.float16: TR_F16, torch.bfloat16: TR_BF16, torch.float32: TR_F32, torch.float64: TR_F64,
       torch.int32: TR_U32, torch.uint32: TR_U32, torch.int64: TR_U64, torch.uint64: TR_U64}


class TrError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class tr_map_desc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("deg_p", ctypes.c_int32), ("deg_q", ctypes.c_int32),
                ("iters", ctypes.c_int32), ("coef_p", ctypes.c_void_p), ("coef_q", ctypes.c_void_p)]


class tr_exec(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("workspace", ctypes.c_void_p), ("workspace_bytes", ctypes.c_size_t),
                ("wait_timeout_us", ctypes.c_uint32), ("reserved", ctypes.c_int32),
                ("debug_stall_tile", ctypes.c_int64)]


_lib = None
_lock = threading.Lock()

_P, _I32, _I64, _U32, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_size_t
_E = ctypes.POINTER(tr_exec)
_M = ctypes.POINTER(tr_map_desc)
SIGNATURES = {
    "tr_status_string": ([_I32], ctypes.c_char_p),
    "tr_last_error": ([], ctypes.c_char_p),
    "tr_launch_count": ([], ctypes.c_uint64),
    "tr_workspace_init": ([_P, _SZ, _P], _I32),
    "tr_check": ([_E], _I32),
    "tr_map": ([_M, _P, _I32, _P, _I32, _I64, _E], _I32),
    "tr_reduce_workspace_size": ([_I64, _I32, ctypes.POINTER(_SZ)], _I32),
    "tr_reduce": ([_M, _P, _I32, _I64, _U32, _P, _I32, _P, _P, _E], _I32),
    "tr_segmented_reduce_workspace_size": ([_I64, _I64, _I32, ctypes.POINTER(_SZ)], _I32),
    "tr_segmented_reduce": ([_M, _P, _I32, _I64, _P, _I64, _U32, _P, _I32, _P, _P, _E], _I32),
    "tr_segmented_reduce_host": ([_M, _P, _I32, _I64, _P, _I64, _U32, _P, _I32, _P, _P, _P, _P, _P, _P, _P, _E],
                                 _I32),
    "tr_scan_workspace_size": ([_I64, _I32, _I32, ctypes.POINTER(_SZ)], _I32),
    "tr_scan": ([_M, _P, _I32, _P, _I32, _I64, _P, _E], _I32),
    "tr_scan_noalloc": ([_M, _P, _I32, _P, _I32, _I64, _P, _P, _P], _I32),
    "tr_scan_reduce": ([_M, _P, _I32, _P, _I32, _I64, _I32, _P, _U32, _P, _I32, _P, _P, _E], _I32),
    "tr_batched_plan_create": ([_I64, _P, _P, _M, _I32, _U32, _P, _P, _P, _I32, _P, ctypes.POINTER(_P)], _I32),
    "tr_batched_run": ([_P, _P], _I32),
    "tr_batched_run_unbatched": ([_P, _I32, _P], _I32),
    "tr_batched_plan_describe": ([_P], ctypes.c_char_p),
    "tr_batched_plan_destroy": ([_P], _I32),
    "tr_vandermonde_workspace_size": ([_I64, _I64, ctypes.POINTER(_SZ)], _I32),
    "tr_vandermonde": ([_P, _I64, _P, _I32, _I64, _I32, _P, _I32, _P, _P, _P, _E], _I32),
}


def lib() -> ctypes.CDLL:
    """The loaded libtr.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"{LIB_PATH} is missing: run `python -m paper_2309_03912_b300.build`")
            L = ctypes.CDLL(LIB_PATH)
            for name, (args, res) in SIGNATURES.items():
                fn = getattr(L, name)
                fn.argtypes = args
                fn.restype = res
            _lib = L
    return _lib


def _check(st: int) -> None:
    if st != 0:
        raise TrError(st, lib().tr_last_error().decode())


def dtype_of(t: torch.Tensor) -> int:
    try:
        return _DT[t.dtype]
    except KeyError:
        raise TrError(3, f"unsupported tensor dtype {t.dtype}") from None


def _ptr(t) -> int | None:
    if t is None:
        return None
    if isinstance(t, int):
        return t
    return t.data_ptr()


class MapDesc:
    """ctypes descriptor of a map dict; keeps its coefficient arrays alive."""

    def __init__(self, m: dict):
        cp = [float(c) for c in m.get("cp", [0.0])]
        cq = [float(c) for c in m.get("cq", [1.0])]
        self._cp = (ctypes.c_double * len(cp))(*cp)
        self._cq = (ctypes.c_double * len(cq))(*cq)
        self.c = tr_map_desc(MAP_KINDS[m["kind"]], len(cp) - 1, len(cq) - 1, int(m.get("iters", 0)),
                             ctypes.addressof(self._cp), ctypes.addressof(self._cq))

    def ref(self):
        return ctypes.byref(self.c)


def make_exec(workspace: torch.Tensor | None = None, stream: torch.cuda.Stream | None = None,
              wait_timeout_us: int = 0, debug_stall_tile: int = -1) -> tr_exec:
    s = stream if stream is not None else torch.cuda.current_stream()
    ws = _ptr(workspace) if workspace is not None else None
    nb = workspace.numel() * workspace.element_size() if workspace is not None else 0
    return tr_exec(s.cuda_stream, ws, nb, wait_timeout_us, 0, debug_stall_tile)


def workspace(nbytes: int, device="cuda") -> torch.Tensor:
    """A zero-filled workspace of at least nbytes (torch allocations are 256-byte aligned)."""
    return torch.zeros(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---- workspace sizes -------------------------------------------------------------

def tr_reduce_workspace_size(n: int, xt: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tr_reduce_workspace_size(n, xt, ctypes.byref(b)))
    return b.value


def tr_segmented_reduce_workspace_size(n: int, n_seg: int, xt: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tr_segmented_reduce_workspace_size(n, n_seg, xt, ctypes.byref(b)))
    return b.value


def tr_scan_workspace_size(n: int, xt: int, yt: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tr_scan_workspace_size(n, xt, yt, ctypes.byref(b)))
    return b.value


# ---- entry points ------------------------------------------------------------------

def tr_launch_count() -> int:
    """Kernels the library has enqueued in this process so far."""
    return int(lib().tr_launch_count())


def tr_workspace_init(ws: torch.Tensor, stream=None) -> None:
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().tr_workspace_init(_ptr(ws), ws.numel() * ws.element_size(), s))


def tr_check(ex: tr_exec) -> None:
    _check(lib().tr_check(ctypes.byref(ex)))


def tr_map(m: dict, x: torch.Tensor, y: torch.Tensor, ex: tr_exec | None = None) -> None:
    ex = ex or make_exec()
    md = MapDesc(m)
    _check(lib().tr_map(md.ref(), _ptr(x), dtype_of(x), _ptr(y), dtype_of(y), x.numel(), ctypes.byref(ex)))


def tr_reduce(m: dict, x: torch.Tensor, ops: int, out_sum, out_min, out_max, ex: tr_exec,
              n: int | None = None) -> None:
    md = MapDesc(m)
    st = dtype_of(out_sum) if out_sum is not None else TR_NONE
    _check(lib().tr_reduce(md.ref(), _ptr(x), dtype_of(x), x.numel() if n is None else n, ops, _ptr(out_sum), st,
                           _ptr(out_min), _ptr(out_max), ctypes.byref(ex)))


def tr_segmented_reduce(m: dict, x: torch.Tensor, offsets: torch.Tensor, ops: int, sums, mins, maxs,
                        ex: tr_exec) -> None:
    md = MapDesc(m)
    st = dtype_of(sums) if sums is not None else TR_NONE
    _check(lib().tr_segmented_reduce(md.ref(), _ptr(x), dtype_of(x), x.numel(), _ptr(offsets), offsets.numel() - 1,
                                     ops, _ptr(sums), st, _ptr(mins), _ptr(maxs), ctypes.byref(ex)))


def tr_scan(m: dict, x: torch.Tensor, y: torch.Tensor, ex: tr_exec, carry_in: torch.Tensor | None = None) -> None:
    md = MapDesc(m)
    _check(lib().tr_scan(md.ref(), _ptr(x), dtype_of(x), _ptr(y), dtype_of(y), x.numel(), _ptr(carry_in),
                         ctypes.byref(ex)))


def tr_scan_reduce(m: dict, x: torch.Tensor, y: torch.Tensor, ex: tr_exec, exclusive: bool = False,
                   carry_in: torch.Tensor | None = None, ops: int = 0, out_sum=None, out_min=None,
                   out_max=None) -> None:
    """Inclusive or exclusive scan of f(x) into y, with sum / min / max of f from the same pass."""
    md = MapDesc(m)
    st = dtype_of(out_sum) if out_sum is not None else TR_NONE
    _check(lib().tr_scan_reduce(md.ref(), _ptr(x), dtype_of(x), _ptr(y), dtype_of(y), x.numel(), int(exclusive),
                                _ptr(carry_in), ops, _ptr(out_sum), st, _ptr(out_min), _ptr(out_max),
                                ctypes.byref(ex)))


def tr_scan_noalloc(m: dict, x: torch.Tensor, y: torch.Tensor, status: torch.Tensor | None = None,
                    carry_in: torch.Tensor | None = None, stream=None) -> None:
    """tr_scan without a workspace (fixed library scratch, n <= 2^26)."""
    md = MapDesc(m)
    s = (stream or torch.cuda.current_stream()).cuda_stream
    _check(lib().tr_scan_noalloc(md.ref(), _ptr(x), dtype_of(x), _ptr(y), dtype_of(y), x.numel(), _ptr(carry_in),
                                 _ptr(status), s))


class BatchPlan:
    """A tr_batched plan over a list of device tensors (one storage dtype: f32, f16 or bf16), one map dict each."""

    def __init__(self, xs, maps, sums, mins, maxs, ops: int = TR_SUM | TR_MIN | TR_MAX, autotune: bool = False,
                 stream=None):
        n = len(xs)
        self._keep = [MapDesc(m) for m in maps]
        descs = (tr_map_desc * n)(*[d.c for d in self._keep])
        ptrs = (ctypes.c_void_p * n)(*[x.data_ptr() for x in xs])
        lens = (ctypes.c_int64 * n)(*[x.numel() for x in xs])
        xt = dtype_of(xs[0]) if n else TR_F32
        self._refs = (xs, sums, mins, maxs)
        self.handle = ctypes.c_void_p()
        s = (stream or torch.cuda.current_stream()).cuda_stream
        _check(lib().tr_batched_plan_create(n, ptrs, lens, descs, xt, ops, _ptr(sums), _ptr(mins), _ptr(maxs),
                                            int(autotune), s, ctypes.byref(self.handle)))

    def describe(self) -> str:
        return lib().tr_batched_plan_describe(self.handle).decode()

    def run(self, stream=None) -> None:
        _check(lib().tr_batched_run(self.handle, (stream or torch.cuda.current_stream()).cuda_stream))

    def run_unbatched(self, use_graph: bool = False, stream=None) -> None:
        _check(lib().tr_batched_run_unbatched(self.handle, int(use_graph),
                                              (stream or torch.cuda.current_stream()).cuda_stream))

    def close(self) -> None:
        if self.handle:
            lib().tr_batched_plan_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def tr_vandermonde_workspace_size(m: int, npoly: int) -> int:
    b = ctypes.c_size_t(0)
    _check(lib().tr_vandermonde_workspace_size(m, npoly, ctypes.byref(b)))
    return b.value


def tr_vandermonde(x: torch.Tensor, coef: torch.Tensor, y: torch.Tensor | None, precision: int, ex: tr_exec,
                   colsum=None, colmin=None, colmax=None) -> None:
    """Y = V(x) C: x (m,) f32, coef (deg+1, npoly) f32 row-major, y (m, npoly) f32 / bf16 or None; optional
    per-column sum / min / max (npoly f32 each)."""
    yt = dtype_of(y) if y is not None else TR_NONE
    _check(lib().tr_vandermonde(_ptr(x), x.numel(), _ptr(coef), coef.shape[0] - 1, coef.shape[1], precision, _ptr(y),
                                yt, _ptr(colsum), _ptr(colmin), _ptr(colmax), ctypes.byref(ex)))
