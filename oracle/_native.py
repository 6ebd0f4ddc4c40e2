"""Build and load the oracle's C part (the Jacobi eigensolver).

ORACLE / TEST INFRASTRUCTURE ONLY: imported by tests, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the GPU product path.

The shared object is compiled in-tree with the host C compiler on first use
(plain C99, no architecture-specific flags, so the same source builds on x86
and on Arm hosts) and cached under ``oracle/_build``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SRC = os.path.join(_HERE, "jacobi.c")
_SO = os.path.join(_BUILD, "liboracle_jacobi.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``jacobi.c`` into ``_build/liboracle_jacobi.so``; return its path."""
    os.makedirs(_BUILD, exist_ok=True)
    stale = (not os.path.exists(_SO)) or os.path.getmtime(_SO) < os.path.getmtime(_SRC)
    if force or stale:
        cc = os.environ.get("CC", "gcc")
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call([cc, "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            so = ctypes.CDLL(path)
            so.oracle_jacobi_eigh.restype = ctypes.c_int
            so.oracle_jacobi_eigh.argtypes = [
                ctypes.c_int,
                ctypes.POINTER(ctypes.c_double),
                ctypes.POINTER(ctypes.c_double),
                ctypes.POINTER(ctypes.c_double),
                ctypes.c_double,
                ctypes.c_int,
                ctypes.POINTER(ctypes.c_int),
            ]
            _lib = so
    return _lib
