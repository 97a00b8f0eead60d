"""The C interface (include/*.h): the library builds, loads without a GPU,
exports every function the headers declare, and the ctypes structures of the
Python binding have the sizes and field offsets of the C structures."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

import paper_2605_18254_gb300 as srm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = sorted(glob.glob(os.path.join(ROOT, "include", "*.h")))


def declared_functions():
    txt = "".join(open(h).read() for h in HEADERS)
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"\b(srm_[a-z_0-9]+)\s*\(", txt)
    return sorted(set(n for n in names if not n.endswith("_t")))


def test_library_exports_every_declared_function():
    lib = srm.load()
    names = declared_functions()
    assert "srm_init" in names and "srm_run_to_target" in names and "srm_plt_step" in names
    out = subprocess.run(["nm", "-D", "--defined-only", lib._name], capture_output=True,
                         text=True, check=True).stdout
    exported = set(re.findall(r" T (srm_[a-z_0-9]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing


STRUCTS = {
    "srm_radii": srm.srm_radii,
    "srm_params": srm.srm_params,
    "srm_allocator": srm.srm_allocator,
    "srm_step_info": srm.srm_step_info,
    "srm_run_info": srm.srm_run_info,
    "srm_state_info": srm.srm_state_info,
    "srm_timings": srm.srm_timings,
    "srm_job": srm.srm_job,
    "srm_tuning": srm.srm_tuning,
    "srm_plt_params": srm.srm_plt_params,
    "srm_plt_step_info": srm.srm_plt_step_info,
    "srm_plt_run_info": srm.srm_plt_run_info,
}


def test_struct_layouts_match(tmp_path):
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "srm.h"', '#include "srm_platelet.h"',
             "int main(void){"]
    for cname, cls in STRUCTS.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for fname, _ in cls._fields_:
            c_field = "lambda" if fname == "lambda_" else fname
            lines.append(f'printf("{cname}.{fname} %zu\\n", offsetof({cname}, {c_field}));')
    lines.append("return 0;}")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(l.split() for l in subprocess.run([str(exe)], capture_output=True, text=True,
                                                  check=True).stdout.splitlines())
    for cname, cls in STRUCTS.items():
        assert int(got[cname]) == ctypes.sizeof(cls), cname
        for fname, _ in cls._fields_:
            assert int(got[f"{cname}.{fname}"]) == getattr(cls, fname).offset, (cname, fname)


def test_invalid_arguments_are_rejected_without_gpu_work():
    """Argument checks run on the host before any CUDA call."""
    lib = srm.load()
    p = srm.srm_params()
    lib.srm_params_default(ctypes.byref(p))
    p.c_m = 0.01
    r = srm.srm_radii()
    r.kind, r.n, r.mean = srm.RADII_MONO, 10, 0.01
    box = (ctypes.c_double * 3)(1.0, 1.0, 1.0)
    h = ctypes.c_void_p()
    cases = [
        dict(dim=4), dict(phi=1.2), dict(phi=0.0), dict(n=0), dict(c_m=0.0), dict(N_l=0),
        dict(box0=-1.0), dict(precision=16),
    ]
    for c in cases:
        p2 = srm.srm_params.from_buffer_copy(p)
        r2 = srm.srm_radii.from_buffer_copy(r)
        b2 = (ctypes.c_double * 3)(*box)
        if "c_m" in c:
            p2.c_m = c["c_m"]
        if "N_l" in c:
            p2.N_l = c["N_l"]
        if "precision" in c:
            p2.precision = c["precision"]
        if "n" in c:
            r2.n = c["n"]
        if "box0" in c:
            b2[0] = c["box0"]
        st = lib.srm_init(ctypes.byref(h), c.get("dim", 3), b2, ctypes.byref(r2), c.get("phi", 0.3),
                          1, ctypes.byref(p2), None, None)
        assert st == 1, c
        assert srm.srm_last_error()


def test_platelet_arguments_are_rejected_without_gpu_work():
    lib = srm.load()
    p = srm.srm_plt_params()
    lib.srm_plt_params_default(ctypes.byref(p))
    assert p.c_m == 0.0 and p.N_k == p.N_l == p.N_shake == 10 and p.c_r == 0.0
    p.c_m = 0.01
    x = (ctypes.c_double * 6)(0.2, 0.2, 0.2, 0.7, 0.7, 0.7)
    u = (ctypes.c_double * 6)(0, 0, 1, 1, 0, 0)
    h = ctypes.c_void_p()
    cases = [dict(c_r=1.0), dict(c_r=-0.1), dict(c_m=0.0), dict(N_l=65536), dict(N_k=0), dict(c_w=-1.0),
             dict(a0=0.0), dict(lam_t=0.5), dict(box0=0.1), dict(n=0), dict(x0=1.5)]
    for c in cases:
        p2 = srm.srm_plt_params.from_buffer_copy(p)
        for k in ("c_r", "c_m", "N_l", "N_k", "c_w"):
            if k in c:
                setattr(p2, k, c[k])
        b = (ctypes.c_double * 3)(c.get("box0", 1.0), 1.0, 1.0)
        x2 = (ctypes.c_double * 6)(*x)
        if "x0" in c:
            x2[0] = c["x0"]
        st = lib.srm_plt_init(ctypes.byref(h), b, c.get("n", 2), c.get("a0", 0.02), 0.002, ctypes.addressof(x2),
                              ctypes.addressof(u), 1.0, c.get("lam_t", 1.0), 1, ctypes.byref(p2), None)
        assert st == 1, c
        assert srm.srm_last_error()
    lam = ctypes.c_double()
    box = (ctypes.c_double * 3)(1.0, 2.0, 0.5)
    assert lib.srm_plt_lambda_for_density(box, 100, 0.1, 0.01, 2.0, ctypes.byref(lam)) == 0
    assert 100 * (2 * lam.value * 0.11) ** 3 == pytest.approx(2.0, rel=1e-14)  # Eq. 1 with V = 1
    assert lib.srm_plt_lambda_for_density(box, 0, 0.1, 0.01, 2.0, ctypes.byref(lam)) == 1
