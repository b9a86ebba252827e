"""ctypes loading of the in-tree native libraries.

Loading fails loudly (ImportError with the path) when a library has not been
built: there is no fallback implementation of any step.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIBDIR = os.path.join(HERE, "_lib")

_lock = threading.Lock()
_libs = {}

c_i32, c_i64, c_vp, c_int = ctypes.c_int32, ctypes.c_int64, ctypes.c_void_p, ctypes.c_int


def _load(name: str) -> ctypes.CDLL:
    with _lock:
        if name in _libs:
            return _libs[name]
        path = os.path.join(LIBDIR, name)
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: run __graft_entry__.build() "
                              f"(python -c 'import __graft_entry__ as g; g.build()')")
        lib = ctypes.CDLL(path)
        _libs[name] = lib
        return lib


def factor_lib() -> ctypes.CDLL:
    lib = _load("libscfactor.so")
    if not getattr(lib, "_typed", False):
        lib.scf_factorize.argtypes = [c_i32, c_vp, c_vp, c_vp, c_i32, c_vp, c_vp, c_i32, ctypes.POINTER(c_vp)]
        lib.scf_factorize.restype = c_int
        lib.scf_analyze.argtypes = [c_i32, c_vp, c_vp, c_i32, c_vp, c_vp, c_i32, ctypes.POINTER(c_vp)]
        lib.scf_analyze.restype = c_int
        lib.scf_numeric.argtypes = [c_vp, c_vp, c_vp]
        lib.scf_numeric.restype = c_int
        lib.scf_nnz.argtypes = [c_vp]
        lib.scf_nnz.restype = c_i64
        lib.scf_export.argtypes = [c_vp, c_vp, c_vp, c_vp, c_vp]
        lib.scf_export.restype = c_int
        lib.scf_free.argtypes = [c_vp]
        lib.scf_free.restype = None
        lib.scf_implicit_apply.argtypes = [c_i32, c_vp, c_i64, c_vp, c_vp, c_i32]
        lib.scf_implicit_apply.restype = c_int
        lib.scf_implicit_plan.argtypes = [c_i32, c_vp, c_i64, ctypes.POINTER(c_vp)]
        lib.scf_implicit_plan.restype = c_int
        lib.scf_implicit_run.argtypes = [c_vp, c_vp, c_vp, c_i32]
        lib.scf_implicit_run.restype = c_int
        lib.scf_solve.argtypes = [c_i32, c_vp, c_vp, c_vp, c_vp, c_vp]
        lib.scf_solve.restype = c_int
        lib.scf_implicit_free.argtypes = [c_vp]
        lib.scf_implicit_free.restype = None
        lib._typed = True
    return lib


def sc_lib() -> ctypes.CDLL:
    lib = _load("libsc.so")
    if not getattr(lib, "_typed", False):
        from . import abi
        abi.declare(lib)
        lib._typed = True
    return lib


def pipe_lib() -> ctypes.CDLL:
    sc_lib()
    factor_lib()
    lib = _load("libscpipe.so")
    if not getattr(lib, "_typed", False):
        from . import abi
        abi.declare_pipeline(lib)
        lib._typed = True
    return lib


def dense_lib() -> ctypes.CDLL:
    lib = _load("libsc_dense.so")
    if not getattr(lib, "_typed", False):
        from . import abi
        abi.declare_dense(lib)
        lib._typed = True
    return lib
