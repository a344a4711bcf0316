"""The C-ABI library loads and exports every symbol that include/dg.h declares
(no compute call: runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "dg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src)))


def test_header_symbols_exported():
    from paper_2409_09620_gb300 import build, native
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # the binding declares a signature for every exported entry point
    assert set(names) <= set(native.SIGNATURES), set(names) - set(native.SIGNATURES)


def test_no_oracle_in_product():
    """The product package never imports or links the oracle."""
    pkg = os.path.join(ROOT, "paper_2409_09620_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in txt.lower() or f == "workloads.py", f


def test_mesh_create_rejects_bad_input_before_any_device_call():
    """dg_mesh_create validates on the host first: bad input returns its
    status and a message without touching the device (so it runs here)."""
    from paper_2409_09620_gb300 import build
    lib = ctypes.CDLL(build.build())
    lib.dg_mesh_create.restype = ctypes.c_int32
    lib.dg_mesh_create.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]
    lib.dg_last_error.restype = ctypes.c_char_p
    xy = (ctypes.c_double * 6)(0, 0, 1, 0, 0, 1)
    cw = (ctypes.c_int32 * 3)(0, 2, 1)
    ccw = (ctypes.c_int32 * 3)(0, 1, 2)
    walls = (ctypes.c_int8 * 3)(1, 1, 1)
    out = ctypes.c_void_p(1)
    assert lib.dg_mesh_create(3, xy, 1, ccw, None, walls, None) == -1              # DG_EINVAL: out NULL
    assert lib.dg_mesh_create(3, xy, 0, ccw, None, walls, ctypes.byref(out)) == -1 and out.value is None
    assert b"empty mesh" in lib.dg_last_error()
    assert lib.dg_mesh_create(3, xy, 1, cw, None, walls, ctypes.byref(out)) == -2  # DG_EMESH
    assert b"counter-clockwise" in lib.dg_last_error() and out.value is None
    assert lib.dg_mesh_create(3, xy, 1, ccw, None, None, ctypes.byref(out)) == -2
    assert b"no valid tag" in lib.dg_last_error()
