"""Loader of the platelet kernel specification (plt_kernel_spec.c).

TEST INFRASTRUCTURE ONLY.  The specification is the binary32 contact
decision exactly as the CUDA kernel evaluates it (threshold widened by
SLACK a); it is built here with plain gcc and handed to the reference's
sweeps (``oracle.PlateletSystem(..., contact=address())``) so that whole GPU
sweeps can be compared bit for bit.  The reference's own decision stays the
binary64 one; the tests pin this specification to it one-sidedly.
"""
import ctypes
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "plt_kernel_spec.c")
BUILD = os.path.join(HERE, "_build")
SO = os.path.join(BUILD, "libplt_kernel_spec.so")
SLACK = 2.0 ** -16  # threshold widening of the kernel, in units of the disk radius

_lib = None
_lock = threading.Lock()


def lib():
    global _lib
    with _lock:
        if _lib is None:
            os.makedirs(BUILD, exist_ok=True)
            if not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
                tmp = SO + f".{os.getpid()}.tmp"
                subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                                       "-o", tmp, SRC, "-lm"])
                os.replace(tmp, SO)
            L = ctypes.CDLL(SO)
            P = ctypes.POINTER(ctypes.c_double)
            L.spec_plt_collide32.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double]
            L.spec_plt_collide32.restype = ctypes.c_int
            _lib = L
    return _lib


def _v3(v):
    return np.ascontiguousarray(v, dtype=np.float64).reshape(3)


def collide32(dj, ni, nj, a, t) -> int:
    P = ctypes.POINTER(ctypes.c_double)
    d, u, v = _v3(dj), _v3(ni), _v3(nj)
    return int(lib().spec_plt_collide32(d.ctypes.data_as(P), u.ctypes.data_as(P), v.ctypes.data_as(P), a, t))


def address() -> int:
    """Address of the specification's contact predicate (for the reference's
    contact hook)."""
    return ctypes.cast(lib().spec_plt_collide32, ctypes.c_void_p).value
