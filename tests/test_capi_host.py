"""Host-side checks of the C ABI (CPU only, no kernel is launched).

* libtr.so loads and exports every function declared in include/*.h;
* argument validation rejects bad calls before any CUDA work;
* workspace-size queries are pure host arithmetic.
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        src = re.sub(r"//[^\n]*", "", src)
        for m in re.finditer(r"\b(tr_[a-z0-9_]+)\s*\(", src):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def L():
    from paper_2309_03912_b300 import binding, build
    build.build()
    return binding.lib()


def test_exports_every_declared_symbol(L):
    names = _declared_functions()
    assert {"tr_map", "tr_reduce", "tr_scan", "tr_segmented_reduce"} <= set(names)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, f"declared but not exported: {missing}"


def test_status_strings(L):
    for s in range(8):
        assert L.tr_status_string(s).decode().startswith("TR_")


def test_validation_rejects_before_launch(L):
    from paper_2309_03912_b300 import binding as B
    ex = B.tr_exec(None, None, 0, 0, 0, -1)
    E = ctypes.byref(ex)
    md = B.MapDesc({"kind": "horner", "cp": [1.0, 2.0]})
    mx = B.MapDesc({"kind": "xorshift32"})
    assert L.tr_reduce(None, None, B.TR_F32, 0, B.TR_SUM, None, B.TR_F32, None, None, E) == 1      # NULL map
    assert L.tr_reduce(md.ref(), None, B.TR_F32, -1, B.TR_SUM, None, B.TR_F32, None, None, E) == 1  # n < 0
    assert L.tr_reduce(md.ref(), None, B.TR_F32, 0, 0, None, B.TR_F32, None, None, E) == 1          # empty ops
    assert L.tr_reduce(mx.ref(), None, B.TR_F32, 0, B.TR_SUM, 8, B.TR_F32, None, None, E) == 3      # mixer on float
    assert L.tr_reduce(md.ref(), None, B.TR_U32, 0, B.TR_SUM, 8, B.TR_U64, None, None, E) == 3      # float map on u32
    assert L.tr_reduce(md.ref(), None, B.TR_F32, 0, B.TR_SUM, 8, B.TR_U64, None, None, E) == 3      # sum dtype
    assert L.tr_reduce(md.ref(), None, B.TR_F32, 0, B.TR_SUM, 8, B.TR_F32, None, None, E) == 4      # no workspace
    assert "workspace" in L.tr_last_error().decode()
    assert L.tr_reduce(md.ref(), None, B.TR_F32, 0, B.TR_SUM, 6, B.TR_F64, None, None, E) == 2      # misaligned sum
    bad = B.tr_map_desc(2, 40, 0, 0, None, None)
    assert L.tr_map(ctypes.byref(bad), None, B.TR_F32, None, B.TR_F32, 0, E) == 1                   # degree > 31
    assert L.tr_map(md.ref(), 64, B.TR_F16, 128, B.TR_F16, 4, E) == 3                               # yt != compute
    assert L.tr_map(md.ref(), 64, B.TR_F32, 68, B.TR_F32, 4, E) == 1                                # partial overlap
    assert L.tr_scan(md.ref(), 64, B.TR_F32, 128, B.TR_F64, 4, None, E) == 3                        # scan dtypes
    assert L.tr_segmented_reduce(md.ref(), None, B.TR_F32, 0, None, -1, B.TR_SUM, None, B.TR_F64, None, None,
                                 E) == 1                                                            # n_seg < 0
    assert L.tr_segmented_reduce(md.ref(), None, B.TR_F64, 0, 8, 1, B.TR_SUM, 8, B.TR_F64, None, None,
                                 E) == 3                                                            # f64 segments


def test_workspace_sizes(L):
    from paper_2309_03912_b300 import binding as B
    assert B.tr_reduce_workspace_size(1 << 20, B.TR_F32) >= 256
    s1 = B.tr_scan_workspace_size(1 << 20, B.TR_U32, B.TR_U32)
    s2 = B.tr_scan_workspace_size(1 << 28, B.TR_U32, B.TR_U32)
    assert s2 > s1 > 256
    assert B.tr_segmented_reduce_workspace_size(1 << 28, 65536, B.TR_F32) >= 256
