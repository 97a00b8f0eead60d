"""Python binding of the SRM CUDA library (include/srm.h).

Argument marshalling only: every step of the method runs in the CUDA
kernels of ``libsrm.so``.  Functions carry the names of the C interface
(``srm_init``, ``srm_step``, ``srm_run_to_target``, ``srm_certify``,
``srm_positions``, ...); the ``Rve`` class wraps one handle.  PyTorch supplies
the CUDA stream and, by default, device memory through its caching allocator.

The library is built in the package tree (``build.py``); loading fails with
an exception if it cannot be built or loaded -- there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading
from ctypes import (CFUNCTYPE, POINTER, Structure, c_char_p, c_double, c_int32, c_int64,
                    c_size_t, c_uint64, c_void_p)

import numpy as np

from . import build as _build

__all__ = ["SrmError", "Rve", "load", "srm_init", "srm_step", "srm_run_to_target", "srm_certify",
           "srm_positions", "srm_overlap_pairs", "srm_sweep", "srm_set_scale", "srm_get_state",
           "srm_nearest", "srm_rdf", "srm_voronoi_lvf", "srm_tuning",
           "srm_destroy", "srm_last_error", "srm_set_timing", "srm_get_timings",
           "srm_certify_noalloc", "srm_save", "srm_load", "srm_job_footprint", "make_job", "Batch",
           "PREC_F64", "PREC_F32", "Platelets", "srm_plt_lambda_for_density", "srm_plt_collide_pairs"]

PREC_F64, PREC_F32 = 64, 32
RADII_EXPLICIT, RADII_MONO, RADII_LOGNORMAL = 0, 1, 2
INIT_RSA_UNIFORM, INIT_RSA_CLUSTERED, INIT_EXPLICIT = 0, 1, 2

STATUS = {0: "SRM_OK", 1: "SRM_E_ARG", 2: "SRM_E_NOMEM", 3: "SRM_E_CUDA",
          4: "SRM_E_NOT_CONVERGED", 5: "SRM_E_DEVICE_TIMEOUT", 6: "SRM_E_CERTIFY_FAILED",
          7: "SRM_E_STATE", 8: "SRM_E_INIT"}


class SrmError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS.get(status, status)}: {message}")
        self.status = status
        self.message = message


class srm_radii(Structure):
    _fields_ = [("kind", c_int32), ("n", c_int64), ("r", c_void_p), ("mean", c_double),
                ("sd", c_double), ("lo", c_double), ("hi", c_double)]


class srm_params(Structure):
    _fields_ = [("c_w", c_double), ("c_m", c_double), ("N_k", c_int32), ("N_l", c_int32),
                ("N_shake", c_int32), ("precision", c_int32), ("init", c_int32),
                ("n_clusters", c_int32), ("cluster_sigma", c_double), ("f0", c_double),
                ("init_pos", c_void_p), ("lambda0", c_double), ("lambda_t", c_double),
                ("guard", c_double), ("sweep0", c_uint64), ("wait_limit", c_int32),
                ("images", c_int32)]


ALLOC_FN = CFUNCTYPE(c_void_p, c_void_p, c_size_t, c_void_p)
FREE_FN = CFUNCTYPE(None, c_void_p, c_void_p, c_void_p)


class srm_allocator(Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", c_void_p)]


class srm_step_info(Structure):
    _fields_ = [("result", c_int32), ("k_sweeps", c_int32), ("shake_sweeps", c_int32),
                ("overlapping", c_int64), ("phi", c_double), ("lambda_", c_double),
                ("sweep", c_uint64)]


class srm_run_info(Structure):
    _fields_ = [("iterations", c_int64), ("accepted", c_int64), ("shaken", c_int64),
                ("sweeps", c_int64), ("phi", c_double), ("lambda_", c_double), ("sweep", c_uint64)]


class srm_state_info(Structure):
    _fields_ = [("dim", c_int32), ("precision", c_int32), ("n", c_int64), ("lambda_", c_double),
                ("lambda_t", c_double), ("phi", c_double), ("phi_t", c_double),
                ("sweep", c_uint64), ("iterations", c_int64), ("accepted", c_int64),
                ("shaken", c_int64), ("sweeps", c_int64), ("done", c_int32),
                ("grid", c_int32 * 3), ("kernel_launches", c_int64), ("pairs_sweep", c_uint64),
                ("pairs_check", c_uint64), ("stage_overflow", c_uint64), ("stage_capacity", c_int32),
                ("check_kernel", c_int32), ("trials", c_uint64), ("pairs_alg5", c_uint64),
                ("near_fallback", c_uint64)]


class srm_job(Structure):
    _fields_ = [("dim", c_int32), ("box", c_double * 3), ("radii", srm_radii), ("phi_t", c_double),
                ("seed", c_uint64), ("params", srm_params)]


class srm_tuning(Structure):
    _fields_ = [("sweep_blocks_per_sm", c_int32), ("stage_capacity", c_int32), ("candidates", c_int32),
                ("sweep_path", c_int32), ("ns_per_particle_sweep", c_double)]


class srm_plt_params(Structure):
    _fields_ = [("c_w", c_double), ("c_m", c_double), ("c_r", c_double), ("N_k", c_int32), ("N_l", c_int32),
                ("N_shake", c_int32), ("wait_limit", c_int32), ("sweep0", c_uint64), ("images", c_int32),
                ("sweep_kernel", c_int32)]


class srm_plt_step_info(Structure):
    _fields_ = [("result", c_int32), ("k_sweeps", c_int32), ("shake_sweeps", c_int32), ("reserved", c_int32),
                ("colliding", c_int64), ("moves", c_int64), ("lambda_", c_double), ("rho", c_double),
                ("sweep", c_uint64)]


class srm_plt_run_info(Structure):
    _fields_ = [("iterations", c_int64), ("accepted", c_int64), ("shaken", c_int64), ("sweeps", c_int64),
                ("moves", c_int64), ("lambda_", c_double), ("rho", c_double), ("converged", c_int32),
                ("reserved", c_int32)]


class srm_timings(Structure):
    _fields_ = [("ms_bin", c_double), ("ms_sweep", c_double), ("ms_check", c_double),
                ("ms_control", c_double), ("supersteps", c_int64), ("sweep_launches", c_int64),
                ("check_launches", c_int64)]


_lib = None
_lock = threading.Lock()
H = c_void_p


def load() -> ctypes.CDLL:
    """Build (if stale) and load libsrm.so; raises if either fails."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            lib = ctypes.CDLL(path, mode=ctypes.RTLD_GLOBAL)
            sig = {
                "srm_params_default": ([POINTER(srm_params)], None),
                "srm_init": ([POINTER(H), c_int32, POINTER(c_double), POINTER(srm_radii), c_double,
                              c_uint64, POINTER(srm_params), c_void_p, POINTER(srm_allocator)],
                             c_int32),
                "srm_step": ([H, POINTER(srm_step_info)], c_int32),
                "srm_run_to_target": ([H, c_int64, POINTER(srm_run_info)], c_int32),
                "srm_certify": ([H, POINTER(c_int64), POINTER(c_double), POINTER(c_double)],
                                c_int32),
                "srm_positions": ([H, c_void_p, c_void_p], c_int32),
                "srm_overlap_pairs": ([H, c_void_p, c_int64, POINTER(c_int64)], c_int32),
                "srm_nearest": ([H, c_void_p, c_void_p, c_void_p], c_int32),
                "srm_rdf": ([H, c_double, c_int32, c_void_p, c_void_p], c_int32),
                "srm_voronoi_lvf": ([H, c_void_p, c_void_p, c_void_p], c_int32),
                "srm_sweep": ([H, c_int32, POINTER(c_int64)], c_int32),
                "srm_set_scale": ([H, c_double], c_int32),
                "srm_get_state": ([H, POINTER(srm_state_info)], c_int32),
                "srm_autotune": ([H, c_int32, POINTER(srm_tuning)], c_int32),
                "srm_set_tuning": ([H, POINTER(srm_tuning)], c_int32),
                "srm_get_tuning": ([H, POINTER(srm_tuning)], c_int32),
                "srm_batch_autotune": ([H, c_int32, POINTER(srm_tuning)], c_int32),
                "srm_batch_set_tuning": ([H, POINTER(srm_tuning)], c_int32),
                "srm_batch_get_tuning": ([H, POINTER(srm_tuning)], c_int32),
                "srm_destroy": ([H], None),
                "srm_set_timing": ([H, c_int32], c_int32),
                "srm_save": ([H, c_void_p, POINTER(c_size_t)], c_int32),
                "srm_load": ([POINTER(H), c_void_p, c_size_t, c_void_p, POINTER(srm_allocator)], c_int32),
                "srm_batch_create": ([POINTER(H), POINTER(srm_job), c_int32, c_void_p,
                                      POINTER(srm_allocator)], c_int32),
                "srm_batch_create_slots": ([POINTER(H), c_int32, c_int64, c_int64, c_int32, c_int32, c_int32,
                                            c_void_p, POINTER(srm_allocator)], c_int32),
                "srm_job_footprint": ([POINTER(srm_job), POINTER(c_int64), POINTER(c_int64)], c_int32),
                "srm_batch_admit": ([H, c_int32, POINTER(srm_job)], c_int32),
                "srm_batch_advance": ([H, c_int32], c_int32),
                "srm_batch_run": ([H, c_int64], c_int32),
                "srm_batch_poll": ([H, POINTER(c_int32), c_int32, POINTER(c_int32)], c_int32),
                "srm_batch_release": ([H, c_int32], c_int32),
                "srm_batch_size": ([H], c_int32),
                "srm_batch_state": ([H, c_int32, POINTER(srm_state_info)], c_int32),
                "srm_batch_positions": ([H, c_int32, c_void_p, c_void_p], c_int32),
                "srm_batch_certify": ([H, c_int32, POINTER(c_int64), POINTER(c_double),
                                       POINTER(c_double)], c_int32),
                "srm_batch_set_timing": ([H, c_int32], c_int32),
                "srm_batch_get_timings": ([H, POINTER(srm_timings)], c_int32),
                "srm_batch_destroy": ([H], None),
                "srm_certify_noalloc": ([c_int32, POINTER(c_double), c_int64, c_void_p, c_void_p,
                                         POINTER(c_int64), POINTER(c_double), c_void_p], c_int32),
                "srm_get_timings": ([H, POINTER(srm_timings)], c_int32),
                "srm_last_error": ([], c_char_p),
                "srm_plt_params_default": ([POINTER(srm_plt_params)], None),
                "srm_plt_lambda_for_density": ([POINTER(c_double), c_int64, c_double, c_double, c_double,
                                                POINTER(c_double)], c_int32),
                "srm_plt_init": ([POINTER(H), POINTER(c_double), c_int64, c_double, c_double, c_void_p, c_void_p,
                                  c_double, c_double, c_uint64, POINTER(srm_plt_params), c_void_p], c_int32),
                "srm_plt_set_params": ([H, POINTER(srm_plt_params)], c_int32),
                "srm_plt_step": ([H, POINTER(srm_plt_step_info)], c_int32),
                "srm_plt_run_to_target": ([H, c_int64, POINTER(srm_plt_run_info)], c_int32),
                "srm_plt_sweeps": ([H, c_int32, POINTER(c_int64)], c_int32),
                "srm_plt_check": ([H, POINTER(c_int64), c_void_p], c_int32),
                "srm_plt_state": ([H, c_void_p, c_void_p, POINTER(c_double), POINTER(c_double), POINTER(c_uint64)],
                                  c_int32),
                "srm_plt_collide_pairs": ([c_void_p, c_void_p, c_void_p, c_int64, c_double, c_double, c_void_p,
                                           c_void_p], c_int32),
                "srm_plt_sweep_stats": ([H, POINTER(c_int64)], c_int32),
                "srm_plt_destroy": ([H], None),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def srm_last_error() -> str:
    return load().srm_last_error().decode()


def _check(st: int):
    if st != 0:
        raise SrmError(st, srm_last_error())


def _as_dict(s: Structure) -> dict:
    out = {}
    for name, _ in s._fields_:
        v = getattr(s, name)
        if hasattr(v, "__len__") and not isinstance(v, (bytes, str)):
            v = list(v)
        out[name.rstrip("_")] = v
    return out


# ---------------------------------------------------------------------------
# C-named functions (thin marshalling)
# ---------------------------------------------------------------------------
def srm_init(dim, box, radii: srm_radii, target_phi, seed, params: srm_params, stream=None,
             allocator: srm_allocator | None = None) -> c_void_p:
    lib = load()
    h = H()
    b = (c_double * 3)(*([float(v) for v in box] + [1.0] * (3 - len(box))))
    _check(lib.srm_init(ctypes.byref(h), int(dim), b, ctypes.byref(radii), float(target_phi),
                        int(seed), ctypes.byref(params), c_void_p(stream or 0),
                        ctypes.byref(allocator) if allocator is not None else None))
    return h


def srm_step(h) -> dict:
    info = srm_step_info()
    _check(load().srm_step(h, ctypes.byref(info)))
    return _as_dict(info)


def srm_run_to_target(h, max_iters: int = 1 << 40) -> dict:
    info = srm_run_info()
    st = load().srm_run_to_target(h, int(max_iters), ctypes.byref(info))
    d = _as_dict(info)
    if st == 4:
        d["converged"] = False
        return d
    _check(st)
    d["converged"] = True
    return d


def srm_certify(h):
    pairs, gap, phi = c_int64(), c_double(), c_double()
    st = load().srm_certify(h, ctypes.byref(pairs), ctypes.byref(gap), ctypes.byref(phi))
    if st not in (0, 6):
        _check(st)
    return int(pairs.value), float(gap.value), float(phi.value)


def srm_positions(h, n: int, dim: int):
    x = np.empty((n, dim), dtype=np.float64)
    r = np.empty(n, dtype=np.float64)
    _check(load().srm_positions(h, x.ctypes.data, r.ctypes.data))
    return x, r


def srm_overlap_pairs(h, cap: int | None = None) -> np.ndarray:
    lib = load()
    n = c_int64()
    if cap is None:
        _check(lib.srm_overlap_pairs(h, None, 0, ctypes.byref(n)))
        cap = int(n.value)
    ij = np.zeros((max(cap, 1), 2), dtype=np.int64)
    _check(lib.srm_overlap_pairs(h, ij.ctypes.data, int(cap), ctypes.byref(n)))
    return ij[:min(int(n.value), cap)].copy()


def srm_nearest(h, n: int):
    """(centre distance, partner id, smallest surface gap) of every particle."""
    d, g = np.zeros(n), np.zeros(n)
    j = np.zeros(n, dtype=np.int64)
    _check(load().srm_nearest(h, d.ctypes.data, j.ctypes.data, g.ctypes.data))
    return d, j, g


def srm_rdf(h, r_max: float, bins: int):
    """(ordered-pair counts per bin, g(r)) of the centres."""
    c = np.zeros(bins, dtype=np.int64)
    g = np.zeros(bins)
    _check(load().srm_rdf(h, float(r_max), int(bins), c.ctypes.data, g.ctypes.data))
    return c, g


def srm_voronoi_lvf(h, n: int, voxels):
    """(voxel counts, local volume fraction) of every particle."""
    M = np.ones(3, dtype=np.int32)
    M[:len(voxels)] = np.asarray(voxels, dtype=np.int32)
    c = np.zeros(n, dtype=np.int64)
    lvf = np.zeros(n)
    _check(load().srm_voronoi_lvf(h, M.ctypes.data, c.ctypes.data, lvf.ctypes.data))
    return c, lvf


def srm_sweep(h, count: int = 1) -> int:
    moved = c_int64()
    _check(load().srm_sweep(h, int(count), ctypes.byref(moved)))
    return int(moved.value)


def srm_set_scale(h, lam: float):
    _check(load().srm_set_scale(h, float(lam)))


def srm_get_state(h) -> dict:
    s = srm_state_info()
    _check(load().srm_get_state(h, ctypes.byref(s)))
    return _as_dict(s)


def srm_set_timing(h, on: bool):
    _check(load().srm_set_timing(h, 1 if on else 0))


def srm_get_timings(h) -> dict:
    t = srm_timings()
    _check(load().srm_get_timings(h, ctypes.byref(t)))
    return _as_dict(t)


def srm_certify_noalloc(dim, box, n, xyz_dev_ptr, radii_dev_ptr, stream=None):
    """Certification of positions and radii held in the caller's device
    buffers (raw device pointers), with no device allocation by the library;
    at most SRM_NOALLOC_MAX_PARTICLES = 32768 particles."""
    b = (c_double * 3)(*([float(v) for v in box] + [1.0] * (3 - len(box))))
    pairs, gap = c_int64(), c_double()
    _check(load().srm_certify_noalloc(int(dim), b, int(n), c_void_p(xyz_dev_ptr),
                                      c_void_p(radii_dev_ptr), ctypes.byref(pairs),
                                      ctypes.byref(gap), c_void_p(stream or 0)))
    return int(pairs.value), float(gap.value)


def srm_destroy(h):
    load().srm_destroy(h)


# ---------------------------------------------------------------------------
# torch plumbing: stream and caching allocator
# ---------------------------------------------------------------------------
def _torch_allocator(device: int):
    import torch

    def _alloc(ctx, nbytes, stream):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), device, int(stream or 0))
        except Exception:
            return None

    def _free(ctx, ptr, stream):
        torch.cuda.caching_allocator_delete(int(ptr))

    fa, ff = ALLOC_FN(_alloc), FREE_FN(_free)
    return srm_allocator(fa, ff, None), (fa, ff)


class Rve:
    """One periodic RVE driven through the C interface.

    radii: array of base radii, or ("mono", r) / ("lognormal", mean, sd, lo, hi) with n.
    init: "rsa" (uniform RSA at f0), "clustered" (RSA with Gaussian cluster
    proposals), or "explicit" (positions given, scale lambda0, default 1).
    """

    def __init__(self, dim, box, radii, target_phi, seed=1, *, n=None, c_m, c_w=0.01, N_k=10,
                 N_l=10, N_shake=10, precision=PREC_F64, init="rsa", positions=None, f0=0.1,
                 n_clusters=0, cluster_sigma=0.0, lambda0=0.0, lambda_t=0.0, guard=4e-6,
                 sweep0=0, wait_limit=0, images=False, stream=None, torch_memory=True):
        import torch
        lib = load()
        self.dim = int(dim)
        rad = srm_radii()
        self._keep = []
        if isinstance(radii, tuple):
            if radii[0] == "mono":
                rad.kind, rad.n, rad.mean = RADII_MONO, int(n), float(radii[1])
            elif radii[0] == "lognormal":
                rad.kind, rad.n = RADII_LOGNORMAL, int(n)
                rad.mean, rad.sd, rad.lo, rad.hi = map(float, radii[1:5])
            else:
                raise ValueError(f"unknown radii spec {radii[0]}")
        else:
            r = np.ascontiguousarray(radii, dtype=np.float64)
            self._keep.append(r)
            rad.kind, rad.n, rad.r = RADII_EXPLICIT, r.size, r.ctypes.data
        self.n = int(rad.n)
        p = srm_params()
        lib.srm_params_default(ctypes.byref(p))
        p.c_w, p.c_m, p.N_k, p.N_l, p.N_shake = c_w, c_m, N_k, N_l, N_shake
        p.precision = int(precision)
        p.init = {"rsa": INIT_RSA_UNIFORM, "clustered": INIT_RSA_CLUSTERED,
                  "explicit": INIT_EXPLICIT}[init]
        if positions is not None:
            x = np.ascontiguousarray(positions, dtype=np.float64)
            self._keep.append(x)
            p.init_pos = x.ctypes.data
        p.f0, p.n_clusters, p.cluster_sigma = f0, n_clusters, cluster_sigma
        p.lambda0, p.lambda_t, p.guard, p.sweep0 = lambda0, lambda_t, guard, sweep0
        p.wait_limit = wait_limit
        p.images = 1 if images else 0
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        alloc = None
        self._cb = None
        if torch_memory:
            alloc, self._cb = _torch_allocator(torch.cuda.current_device())
        self._alloc = alloc
        self.h = srm_init(dim, box, rad, target_phi, seed, p, self.stream, alloc)

    def step(self) -> dict:
        return srm_step(self.h)

    def run_to_target(self, max_iters: int = 1 << 40) -> dict:
        return srm_run_to_target(self.h, max_iters)

    def certify(self):
        return srm_certify(self.h)

    def positions(self):
        return srm_positions(self.h, self.n, self.dim)

    def overlap_pairs(self) -> np.ndarray:
        return srm_overlap_pairs(self.h)

    def autotune(self, supersteps: int = 8) -> dict:
        t = srm_tuning()
        _check(load().srm_autotune(self.h, int(supersteps), ctypes.byref(t)))
        return _as_dict(t)

    def set_tuning(self, sweep_blocks_per_sm: int, stage_capacity: int = 0, sweep_path: int = 0):
        t = srm_tuning(sweep_blocks_per_sm=int(sweep_blocks_per_sm), stage_capacity=int(stage_capacity),
                       sweep_path=int(sweep_path))
        _check(load().srm_set_tuning(self.h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = srm_tuning()
        _check(load().srm_get_tuning(self.h, ctypes.byref(t)))
        return _as_dict(t)

    def nearest(self):
        return srm_nearest(self.h, self.n)

    def rdf(self, r_max: float, bins: int):
        return srm_rdf(self.h, r_max, bins)

    def voronoi_lvf(self, voxels):
        return srm_voronoi_lvf(self.h, self.n, voxels)

    def sweep(self, count: int = 1) -> int:
        return srm_sweep(self.h, count)

    def set_scale(self, lam: float):
        srm_set_scale(self.h, lam)

    def state(self) -> dict:
        return srm_get_state(self.h)

    def set_timing(self, on: bool = True):
        srm_set_timing(self.h, on)

    def timings(self) -> dict:
        return srm_get_timings(self.h)

    def save(self) -> bytes:
        return srm_save(self.h)

    def close(self):
        if getattr(self, "h", None):
            srm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


# ---------------------------------------------------------------------------
# jobs, batches, serving slots, checkpoints
# ---------------------------------------------------------------------------
def make_job(dim, box, radii, target_phi, seed=1, *, n=None, c_m, c_w=0.01, N_k=10, N_l=10,
             N_shake=10, precision=PREC_F32, init="rsa", positions=None, f0=0.1, n_clusters=0,
             cluster_sigma=0.0, lambda0=0.0, lambda_t=0.0, guard=4e-6, sweep0=0):
    """An srm_job; returns (job, keep) where keep holds the arrays it points to."""
    lib = load()
    job = srm_job()
    keep = []
    job.dim = int(dim)
    for a in range(3):
        job.box[a] = float(box[a]) if a < len(box) else 1.0
    if isinstance(radii, tuple):
        if radii[0] == "mono":
            job.radii.kind, job.radii.n, job.radii.mean = RADII_MONO, int(n), float(radii[1])
        else:
            job.radii.kind, job.radii.n = RADII_LOGNORMAL, int(n)
            job.radii.mean, job.radii.sd, job.radii.lo, job.radii.hi = map(float, radii[1:5])
    else:
        r = np.ascontiguousarray(radii, dtype=np.float64)
        keep.append(r)
        job.radii.kind, job.radii.n, job.radii.r = RADII_EXPLICIT, r.size, r.ctypes.data
    job.phi_t = float(target_phi)
    job.seed = int(seed)
    p = job.params
    lib.srm_params_default(ctypes.byref(p))
    p.c_w, p.c_m, p.N_k, p.N_l, p.N_shake = c_w, c_m, N_k, N_l, N_shake
    p.precision = int(precision)
    p.init = {"rsa": INIT_RSA_UNIFORM, "clustered": INIT_RSA_CLUSTERED, "explicit": INIT_EXPLICIT}[init]
    if positions is not None:
        x = np.ascontiguousarray(positions, dtype=np.float64)
        keep.append(x)
        p.init_pos = x.ctypes.data
    p.f0, p.n_clusters, p.cluster_sigma = f0, n_clusters, cluster_sigma
    p.lambda0, p.lambda_t, p.guard, p.sweep0 = lambda0, lambda_t, guard, sweep0
    return job, keep


def srm_job_footprint(job: srm_job):
    n, c = c_int64(), c_int64()
    _check(load().srm_job_footprint(ctypes.byref(job), ctypes.byref(n), ctypes.byref(c)))
    return int(n.value), int(c.value)


class Batch:
    """Many RVEs advanced by the same launches (srm_batch_*).

    Batch(jobs=[...]) loads the jobs; Batch(slots=k, max_particles=, max_cells=)
    creates empty slots for continuous serving (admit / advance / poll / release).
    """

    def __init__(self, jobs=None, *, slots=0, max_particles=0, max_cells=0, dim=0, precision=PREC_F32,
                 stage_capacity=0, stream=None, torch_memory=True):
        import torch
        lib = load()
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        self.stream = int(stream)
        alloc, self._cb = (None, None)
        if torch_memory:
            alloc, self._cb = _torch_allocator(torch.cuda.current_device())
        self._alloc = alloc
        self.h = H()
        self._meta = {}
        if jobs is not None:
            arr = (srm_job * len(jobs))(*[j for j, _ in jobs])
            self._keep = [k for _, k in jobs]
            _check(lib.srm_batch_create(ctypes.byref(self.h), arr, len(jobs), c_void_p(self.stream),
                                        ctypes.byref(alloc) if alloc is not None else None))
            for i, (j, _) in enumerate(jobs):
                self._meta[i] = (int(j.dim), int(j.radii.n))
        else:
            _check(lib.srm_batch_create_slots(ctypes.byref(self.h), int(slots), int(max_particles),
                                              int(max_cells), int(dim), int(precision), int(stage_capacity),
                                              c_void_p(self.stream),
                                              ctypes.byref(alloc) if alloc is not None else None))

    def __len__(self):
        return int(load().srm_batch_size(self.h))

    def admit(self, slot: int, job_keep):
        job, keep = job_keep
        _check(load().srm_batch_admit(self.h, int(slot), ctypes.byref(job)))
        self._meta[int(slot)] = (int(job.dim), int(job.radii.n))

    def advance(self, supersteps: int):
        _check(load().srm_batch_advance(self.h, int(supersteps)))

    def autotune(self, supersteps: int = 8) -> dict:
        t = srm_tuning()
        _check(load().srm_batch_autotune(self.h, int(supersteps), ctypes.byref(t)))
        return _as_dict(t)

    def set_tuning(self, sweep_blocks_per_sm: int, stage_capacity: int = 0, sweep_path: int = 0):
        t = srm_tuning(sweep_blocks_per_sm=int(sweep_blocks_per_sm), stage_capacity=int(stage_capacity),
                       sweep_path=int(sweep_path))
        _check(load().srm_batch_set_tuning(self.h, ctypes.byref(t)))

    def tuning(self) -> dict:
        t = srm_tuning()
        _check(load().srm_batch_get_tuning(self.h, ctypes.byref(t)))
        return _as_dict(t)

    def run(self, max_iters: int = 1 << 40) -> bool:
        st = load().srm_batch_run(self.h, int(max_iters))
        if st == 4:
            return False
        _check(st)
        return True

    def poll(self) -> list:
        cap = max(1, len(self))
        out = (c_int32 * cap)()
        n = c_int32()
        _check(load().srm_batch_poll(self.h, out, cap, ctypes.byref(n)))
        return [int(out[i]) for i in range(n.value)]

    def release(self, slot: int):
        _check(load().srm_batch_release(self.h, int(slot)))

    def state(self, slot: int) -> dict:
        s = srm_state_info()
        _check(load().srm_batch_state(self.h, int(slot), ctypes.byref(s)))
        return _as_dict(s)

    def positions(self, slot: int):
        dim, n = self._meta[int(slot)]
        x = np.empty((n, dim), dtype=np.float64)
        r = np.empty(n, dtype=np.float64)
        _check(load().srm_batch_positions(self.h, int(slot), x.ctypes.data, r.ctypes.data))
        return x, r

    def certify(self, slot: int):
        pairs, gap, phi = c_int64(), c_double(), c_double()
        st = load().srm_batch_certify(self.h, int(slot), ctypes.byref(pairs), ctypes.byref(gap),
                                      ctypes.byref(phi))
        if st not in (0, 6):
            _check(st)
        return int(pairs.value), float(gap.value), float(phi.value)

    def set_timing(self, on: bool = True):
        _check(load().srm_batch_set_timing(self.h, 1 if on else 0))

    def timings(self) -> dict:
        t = srm_timings()
        _check(load().srm_batch_get_timings(self.h, ctypes.byref(t)))
        return _as_dict(t)

    def close(self):
        if getattr(self, "h", None):
            load().srm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def srm_save(h) -> bytes:
    lib = load()
    n = c_size_t()
    _check(lib.srm_save(h, None, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value)
    _check(lib.srm_save(h, buf, ctypes.byref(n)))
    return buf.raw[:n.value]


def srm_load(data: bytes, stream=None, torch_memory=True) -> "Rve":
    """A new Rve handle continuing from a checkpoint."""
    import torch
    lib = load()
    r = Rve.__new__(Rve)
    r._keep = []
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    r.stream = int(stream)
    alloc, r._cb = (None, None)
    if torch_memory:
        alloc, r._cb = _torch_allocator(torch.cuda.current_device())
    r._alloc = alloc
    buf = ctypes.create_string_buffer(data, len(data))
    h = H()
    _check(lib.srm_load(ctypes.byref(h), buf, len(data), c_void_p(r.stream),
                        ctypes.byref(alloc) if alloc is not None else None))
    r.h = h
    st = srm_get_state(h)
    r.dim, r.n = int(st["dim"]), int(st["n"])
    return r


# ---------------------------------------------------------------------------
# Platelets (include/srm_platelet.h): spherodisks with a rotational move
# ---------------------------------------------------------------------------
def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a if shape is None else a.reshape(shape)


def srm_plt_lambda_for_density(box, n, a0, t0, rho) -> float:
    """Scale at which n platelets reach the number density rho of Eq. 1."""
    L = (c_double * 3)(*[float(v) for v in box])
    out = c_double()
    _check(load().srm_plt_lambda_for_density(L, int(n), float(a0), float(t0), float(rho), ctypes.byref(out)))
    return out.value


def srm_plt_collide_pairs(dj, ni, nj, a, t, stream=None) -> np.ndarray:
    """Contact decisions of m platelet pairs (rows of dj, ni, nj) on the GPU."""
    import torch
    dj, ni, nj = _f64(dj, (-1, 3)), _f64(ni, (-1, 3)), _f64(nj, (-1, 3))
    m = dj.shape[0]
    out = np.zeros(m, dtype=np.uint8)
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    _check(load().srm_plt_collide_pairs(dj.ctypes.data, ni.ctypes.data, nj.ctypes.data, m, float(a), float(t),
                                        out.ctypes.data, stream))
    return out


class Platelets:
    """One platelet RVE on the GPU (srm_plt_* of include/srm_platelet.h):
    centres x and unit normals u (n x 3), base sizes a0, t0, scales lambda0
    (start) and lambda_t (target), seed and the SRM parameters with the
    rotation rate c_r."""

    def __init__(self, box, x, u, a0, t0, lambda0, lambda_t, seed, *, c_m, c_w=0.01, c_r=0.0, N_k=10, N_l=10,
                 N_shake=10, wait_limit=0, sweep0=0, images=False, sweep_kernel=0, stream=None):
        import torch
        lib = load()
        self.box = tuple(float(v) for v in box)
        x, u = _f64(x, (-1, 3)), _f64(u, (-1, 3))
        self.n = x.shape[0]
        p = srm_plt_params()
        lib.srm_plt_params_default(ctypes.byref(p))
        p.c_w, p.c_m, p.c_r, p.N_k, p.N_l, p.N_shake = c_w, c_m, c_r, N_k, N_l, N_shake
        p.wait_limit, p.sweep0 = wait_limit, sweep0
        self._images = 1 if images else 0
        self._sweep_kernel = int(sweep_kernel)
        p.images = self._images
        p.sweep_kernel = self._sweep_kernel
        if stream is None:
            stream = torch.cuda.current_stream().cuda_stream
        L = (c_double * 3)(*self.box)
        h = H()
        _check(lib.srm_plt_init(ctypes.byref(h), L, self.n, float(a0), float(t0), x.ctypes.data, u.ctypes.data,
                                float(lambda0), float(lambda_t), int(seed), ctypes.byref(p), stream))
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            load().srm_plt_destroy(self._h)
            self._h = None

    __del__ = close

    def set_params(self, *, c_m, c_w=0.01, c_r=0.0, N_k=10, N_l=10, N_shake=10, wait_limit=0):
        p = srm_plt_params()
        load().srm_plt_params_default(ctypes.byref(p))
        p.c_w, p.c_m, p.c_r, p.N_k, p.N_l, p.N_shake, p.wait_limit = c_w, c_m, c_r, N_k, N_l, N_shake, wait_limit
        p.images = self._images
        p.sweep_kernel = self._sweep_kernel
        _check(load().srm_plt_set_params(self._h, ctypes.byref(p)))

    def step(self) -> dict:
        info = srm_plt_step_info()
        _check(load().srm_plt_step(self._h, ctypes.byref(info)))
        return _as_dict(info)

    def run_to_target(self, max_iters: int = 0) -> dict:
        info = srm_plt_run_info()
        st = load().srm_plt_run_to_target(self._h, int(max_iters), ctypes.byref(info))
        if st not in (0, 4):
            _check(st)
        return _as_dict(info)

    def sweeps(self, count: int) -> int:
        acc = c_int64()
        _check(load().srm_plt_sweeps(self._h, int(count), ctypes.byref(acc)))
        return acc.value

    def sweep_stats(self) -> dict:
        """Sweeps by kernel (block per cell with the staged neighbourhood;
        warp per cell) and cells the block kernel could not stage."""
        out = (c_int64 * 3)()
        _check(load().srm_plt_sweep_stats(self._h, out))
        return {"staged_sweeps": out[0], "warp_sweeps": out[1], "unstaged_cells": out[2]}

    def check(self):
        cnt = c_int64()
        flags = np.zeros(self.n, dtype=np.uint8)
        _check(load().srm_plt_check(self._h, ctypes.byref(cnt), flags.ctypes.data))
        return cnt.value, flags

    def state(self):
        x = np.zeros((self.n, 3))
        u = np.zeros((self.n, 3))
        lam, rho, sw = c_double(), c_double(), c_uint64()
        _check(load().srm_plt_state(self._h, x.ctypes.data, u.ctypes.data, ctypes.byref(lam), ctypes.byref(rho),
                                    ctypes.byref(sw)))
        return x, u, dict(lambda_=lam.value, rho=rho.value, sweep=sw.value)
