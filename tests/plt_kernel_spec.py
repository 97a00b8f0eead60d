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
BUDGET_GAP = 2.0 ** -12  # largest gap (units of a) at which an exhausted bisection may report contact

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
            for f in (L.spec_plt_collide32, L.spec_plt_collide32_reason):
                f.argtypes = [P, P, P, ctypes.c_double, ctypes.c_double]
                f.restype = ctypes.c_int
            _lib = L
    return _lib


def _v3(v):
    return np.ascontiguousarray(v, dtype=np.float64).reshape(3)


def collide32(dj, ni, nj, a, t) -> int:
    P = ctypes.POINTER(ctypes.c_double)
    d, u, v = _v3(dj), _v3(ni), _v3(nj)
    return int(lib().spec_plt_collide32(d.ctypes.data_as(P), u.ctypes.data_as(P), v.ctypes.data_as(P), a, t))


def reason(dj, ni, nj, a, t) -> int:
    """0 separated; 1 a rim point within the widened threshold; 2 contact
    only because a bisection arc stayed undecided (its budget ran out)."""
    P = ctypes.POINTER(ctypes.c_double)
    d, u, v = _v3(dj), _v3(ni), _v3(nj)
    return int(lib().spec_plt_collide32_reason(d.ctypes.data_as(P), u.ctypes.data_as(P), v.ctypes.data_as(P), a, t))


def confirmed_by_reference(oracle, dj, ni, nj, a, t) -> bool:
    """A contact the specification reports and the binary64 reference does
    not must be within the widening of touching (plus the binary32 rounding
    of its inputs: 1.25 SLACK a), or -- when an arc's bisection ran out of
    budget -- a near-contact within BUDGET_GAP a of touching."""
    if oracle.plt_collide(dj, ni, nj, a, t + 0.5 * 1.25 * SLACK * a):
        return True
    return reason(dj, ni, nj, a, t) == 2 and bool(oracle.plt_collide(dj, ni, nj, a, t + 0.5 * BUDGET_GAP * a))


def address() -> int:
    """Address of the specification's contact predicate (for the reference's
    contact hook)."""
    return ctypes.cast(lib().spec_plt_collide32, ctypes.c_void_p).value
