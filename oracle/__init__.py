"""FP64 CPU reference of SRM -- TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded reference of the Swelling and Random Migration
method (Section 2, Algorithms 1-6), written in C (``srm_oracle.c``) and driven
from here through ctypes.  Only the tests, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product library
never does, and the two share no code.  See the header of ``srm_oracle.c``
for the readings of the paper it fixes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "srm_oracle.c")
_SRC_A = os.path.join(_HERE, "srm_analysis.c")
_SRC_P = os.path.join(_HERE, "srm_platelet.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsrm_oracle.so")
_lock = threading.Lock()
_lib = None

P = ctypes.POINTER
_d, _i64, _u64, _int = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64, ctypes.c_int


def build(force: bool = False) -> str:
    """Compile the reference with plain gcc, no FMA contraction, no fast-math."""
    os.makedirs(_BUILD, exist_ok=True)
    srcs = [_SRC, _SRC_A, _SRC_P]
    deps = srcs + [os.path.join(_HERE, "orc_images.h")]
    if force or not os.path.exists(_SO) or any(os.path.getmtime(_SO) < os.path.getmtime(f) for f in deps):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", "-o", tmp] + srcs + ["-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            sig = {
                "orc_philox4x32_10": ([P(ctypes.c_uint32), P(ctypes.c_uint32), P(ctypes.c_uint32)], None),
                "orc_unit_dir": ([_u64, _u64, _u64, _u64, _int, P(_d)], _int),
                "orc_wrap": ([_d, _d], _d),
                "orc_grid": ([_int, P(_d), _d, _d, _d, P(_i64), P(_d)], None),
                "orc_create": ([_int, P(_d), _i64, P(_d), P(_d), _d, _d, _d, _d, _int, _int, _int,
                                _u64, _u64, _int], ctypes.c_void_p),
                "orc_destroy": ([ctypes.c_void_p], None),
                "orc_get_x": ([ctypes.c_void_p, P(_d)], None),
                "orc_set_x": ([ctypes.c_void_p, P(_d)], None),
                "orc_get_lambda": ([ctypes.c_void_p], _d),
                "orc_set_lambda": ([ctypes.c_void_p, _d], None),
                "orc_get_sweep": ([ctypes.c_void_p], _u64),
                "orc_set_margin": ([ctypes.c_void_p, P(_d)], None),
                "orc_set_images": ([ctypes.c_void_p, _int], None),
                "orc_images_verify": ([ctypes.c_void_p, P(_d)], _i64),
                "orc_images_count": ([ctypes.c_void_p], _i64),
                "orc_get_counters": ([ctypes.c_void_p, P(_i64)], None),
                "orc_phi": ([ctypes.c_void_p, _d], _d),
                "orc_lambda_for_phi": ([ctypes.c_void_p, _d], _d),
                "orc_sweep": ([ctypes.c_void_p], _i64),
                "orc_check": ([ctypes.c_void_p, P(ctypes.c_uint8)], _i64),
                "orc_pairs": ([ctypes.c_void_p, P(_i64), _i64], _i64),
                "orc_iterate": ([ctypes.c_void_p, P(_i64)], _int),
                "orc_run": ([ctypes.c_void_p, _i64], _i64),
                "orc_pairs_brute": ([_int, P(_d), _i64, P(_d), P(_d), P(_i64), _i64, P(_d)], _i64),
                "orc_certify": ([_int, P(_d), _i64, P(_d), P(_d), P(_d)], _i64),
                "orc_nn": ([_int, P(_d), _i64, P(_d), P(_d), P(_d), P(_i64), P(_d)], None),
                "orc_rdf": ([_int, P(_d), _i64, P(_d), _d, _int, P(_i64), P(_d)], _i64),
                "orc_voronoi_lvf": ([_int, P(_d), _i64, P(_d), P(_d), P(ctypes.c_int32), P(_i64), P(_d)], None),
                "orc_unit_dir_stream": ([_u64, _u64, _u64, _u64, _int, _int, P(_d)], _int),
                "orc_plt_basis": ([P(_d), P(_d), P(_d)], None),
                "orc_plt_point_disk": ([P(_d), P(_d), P(_d), _d], _d),
                "orc_plt_rim_near_disk": ([P(_d), P(_d), _d, P(_d), P(_d), _d, _d, P(_int)], _int),
                "orc_plt_set_contact": ([ctypes.c_void_p, ctypes.c_void_p], None),
                "orc_plt_set_images": ([ctypes.c_void_p, _int], None),
                "orc_plt_images_verify": ([ctypes.c_void_p], _i64),
                "orc_plt_collide": ([P(_d), P(_d), P(_d), _d, _d], _int),
                "orc_plt_trial": ([_u64, _u64, _u64, _u64, P(_d), _d, _d, P(_d), P(_d), P(_d), P(_d)], None),
                "orc_plt_create": ([P(_d), _i64, P(_d), P(_d), _d, _d, _d, _d, _d, _d, _d, _int, _int, _int,
                                    _u64, _u64], ctypes.c_void_p),
                "orc_plt_destroy": ([ctypes.c_void_p], None),
                "orc_plt_get": ([ctypes.c_void_p, P(_d), P(_d)], None),
                "orc_plt_lambda": ([ctypes.c_void_p], _d),
                "orc_plt_sweep_counter": ([ctypes.c_void_p], _u64),
                "orc_plt_counters": ([ctypes.c_void_p, P(_i64)], None),
                "orc_plt_sweep": ([ctypes.c_void_p], _i64),
                "orc_plt_check": ([ctypes.c_void_p, P(ctypes.c_uint8)], _i64),
                "orc_plt_iterate": ([ctypes.c_void_p, P(_i64)], _int),
                "orc_plt_run": ([ctypes.c_void_p, _i64], _i64),
                "orc_plt_pairs_brute": ([P(_d), _i64, P(_d), P(_d), _d, _d, P(_i64), _i64], _i64),
            }
            for name, (args, res) in sig.items():
                f = getattr(lib, name)
                f.argtypes = args
                f.restype = res
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(P(_d))


def _box3(box, dim):
    L = np.ones(3)
    L[:dim] = np.asarray(box, dtype=np.float64)[:dim]
    return L


def philox4x32_10(ctr, key) -> np.ndarray:
    u32 = ctypes.c_uint32
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    _load().orc_philox4x32_10(c.ctypes.data_as(P(u32)), k.ctypes.data_as(P(u32)), out.ctypes.data_as(P(u32)))
    return out


def unit_dir(seed: int, sweep: int, pid: int, l: int, dim: int):
    u = np.zeros(3)
    m = _load().orc_unit_dir(seed, sweep, pid, l, dim, _dp(u))
    return u[:dim], m


def unit_dir_stream(seed: int, sweep: int, pid: int, l: int, dim: int, stream: int):
    u = np.zeros(3)
    m = _load().orc_unit_dir_stream(seed, sweep, pid, l, dim, stream, _dp(u))
    return u[:dim], m


def wrap(x: float, L: float) -> float:
    return _load().orc_wrap(x, L)


def grid(dim, box, lam, rmax, c_m):
    n = np.zeros(3, dtype=np.int64)
    w = np.zeros(3)
    _load().orc_grid(dim, _dp(_box3(box, dim)), lam, rmax, c_m, n.ctypes.data_as(P(_i64)), _dp(w))
    return n[:dim], w[:dim]


def pairs_brute(dim, box, X, R, cap: int = 1 << 20):
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    ij = np.zeros((cap, 2), dtype=np.int64)
    mg = np.zeros(1)
    cnt = _load().orc_pairs_brute(dim, _dp(_box3(box, dim)), R.size, _dp(X), _dp(R),
                                  ij.ctypes.data_as(P(_i64)), cap, _dp(mg))
    return ij[:min(cnt, cap)].copy(), int(cnt), float(mg[0])


def certify(dim, box, X, R):
    """(colliding pair count, minimum gap S - (R_i + R_j)) by a cell list."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    mg = np.zeros(1)
    cnt = _load().orc_certify(dim, _dp(_box3(box, dim)), R.size, _dp(X), _dp(R), _dp(mg))
    return int(cnt), float(mg[0])


def nn(dim, box, X, R):
    """Nearest neighbours by brute force: (centre distance, partner id,
    smallest surface gap) per particle (Section 3.2, Fig. 4d)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.size
    d, g = np.zeros(n), np.zeros(n)
    j = np.zeros(n, dtype=np.int64)
    _load().orc_nn(dim, _dp(_box3(box, dim)), n, _dp(X), _dp(R), _dp(d), j.ctypes.data_as(P(_i64)), _dp(g))
    return d, j, g


def rdf(dim, box, X, r_max, bins):
    """Radial distribution of the centres: (ordered-pair counts per bin, g)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n = X.shape[0]
    c = np.zeros(bins, dtype=np.int64)
    g = np.zeros(bins)
    _load().orc_rdf(dim, _dp(_box3(box, dim)), n, _dp(X), r_max, bins, c.ctypes.data_as(P(_i64)), _dp(g))
    return c, g


def voronoi_lvf(dim, box, X, R, voxels):
    """Local volume fraction from a discrete periodic Voronoi tessellation on
    the given voxel grid: (voxel counts, LVF) per particle (Section 3.2)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    R = np.ascontiguousarray(R, dtype=np.float64)
    n = R.size
    M = np.ones(3, dtype=np.int32)
    M[:dim] = np.asarray(voxels, dtype=np.int32)[:dim]
    c = np.zeros(n, dtype=np.int64)
    lvf = np.zeros(n)
    _load().orc_voronoi_lvf(dim, _dp(_box3(box, dim)), n, _dp(X), _dp(R), M.ctypes.data_as(P(ctypes.c_int32)),
                            c.ctypes.data_as(P(_i64)), _dp(lvf))
    return c, lvf


class System:
    """One RVE in the reference: P (positions in id order), base radii r,
    scale lambda (R_i = lambda r_i), target scale, and the SRM parameters."""

    def __init__(self, dim, box, x, r, lam=1.0, lam_t=None, target_phi=None, c_w=0.01,
                 c_m=0.01, N_k=10, N_l=10, N_shake=10, seed=1, sweep=0, literal=False, images=False):
        """images: periodicity by explicit image particles instead of the
        minimum image (Section 2; see orc_set_images in srm_oracle.c)."""
        if not 1 <= N_l < (1 << 16):
            raise ValueError("N_l must be in [1, 65535] (the try index takes 16 counter bits)")
        lib = _load()
        self.dim = int(dim)
        self.box = _box3(box, dim)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        self.r = np.ascontiguousarray(r, dtype=np.float64)
        self.n = int(self.r.size)
        self._h = lib.orc_create(self.dim, _dp(self.box), self.n, _dp(x), _dp(self.r), lam,
                                 lam if lam_t is None else lam_t, c_w, c_m, N_k, N_l, N_shake,
                                 seed, sweep, 1 if literal else 0)
        if lam_t is None and target_phi is not None:
            lt = lib.orc_lambda_for_phi(self._h, target_phi)
            lib.orc_destroy(self._h)
            self._h = lib.orc_create(self.dim, _dp(self.box), self.n, _dp(x), _dp(self.r), lam,
                                     lt, c_w, c_m, N_k, N_l, N_shake, seed, sweep,
                                     1 if literal else 0)
        self._margin = None
        self.images = bool(images)
        lib.orc_set_images(self._h, 1 if images else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_destroy(h)
            self._h = None

    @property
    def x(self) -> np.ndarray:
        out = np.zeros(self.n * self.dim)
        _lib.orc_get_x(self._h, _dp(out))
        return out.reshape(self.n, self.dim)

    @x.setter
    def x(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1)
        _lib.orc_set_x(self._h, _dp(v))

    @property
    def lam(self) -> float:
        return _lib.orc_get_lambda(self._h)

    @lam.setter
    def lam(self, v: float):
        _lib.orc_set_lambda(self._h, v)

    @property
    def sweep_counter(self) -> int:
        return int(_lib.orc_get_sweep(self._h))

    def radii(self) -> np.ndarray:
        return self.lam * self.r

    def phi(self, lam=None) -> float:
        return _lib.orc_phi(self._h, self.lam if lam is None else lam)

    def lambda_for_phi(self, phi: float) -> float:
        return _lib.orc_lambda_for_phi(self._h, phi)

    def track_margins(self, on: bool = True):
        self._margin = np.full(self.n, np.inf) if on else None
        _lib.orc_set_margin(self._h, _dp(self._margin) if on else None)

    @property
    def margins(self):
        return None if self._margin is None else self._margin.copy()

    def images_verify(self) -> int:
        """Mismatching padded cells between the image entries kept move by
        move during the last sweep of P and a rebuild from P (0: consistent)."""
        x = np.ascontiguousarray(self.x, dtype=np.float64).reshape(-1)
        return int(_lib.orc_images_verify(self._h, _dp(x)))

    def images_count(self) -> int:
        return int(_lib.orc_images_count(self._h))

    def counters(self) -> dict:
        c = np.zeros(5, dtype=np.int64)
        _lib.orc_get_counters(self._h, c.ctypes.data_as(P(_i64)))
        return dict(iters=int(c[0]), accepted=int(c[1]), shaken=int(c[2]),
                    moves_accepted=int(c[3]), sweeps=int(c[4]))

    def sweep(self) -> int:
        return int(_lib.orc_sweep(self._h))

    def check(self):
        flags = np.zeros(self.n, dtype=np.uint8)
        cnt = _lib.orc_check(self._h, flags.ctypes.data_as(P(ctypes.c_uint8)))
        return int(cnt), flags

    def pairs(self, cap: int = 1 << 20) -> np.ndarray:
        ij = np.zeros((cap, 2), dtype=np.int64)
        cnt = _lib.orc_pairs(self._h, ij.ctypes.data_as(P(_i64)), cap)
        if cnt > cap:
            return self.pairs(int(cnt))
        return ij[:cnt].copy()

    def iterate(self):
        info = np.zeros(3, dtype=np.int64)
        acc = _lib.orc_iterate(self._h, info.ctypes.data_as(P(_i64)))
        return int(acc), dict(k_sweeps=int(info[0]), overlapping=int(info[1]),
                              shake_sweeps=int(info[2]))

    def run(self, max_iters: int = 1 << 40) -> int:
        return int(_lib.orc_run(self._h, max_iters))

    def certify(self):
        return certify(self.dim, self.box[:self.dim], self.x, self.radii())


# ---------------------------------------------------------------------------
# Platelets (spherodisks, Section 3.3): see the header of srm_platelet.c.
# ---------------------------------------------------------------------------
def _v3(v):
    return np.ascontiguousarray(v, dtype=np.float64).reshape(3)


def plt_basis(n):
    e1, e2 = np.zeros(3), np.zeros(3)
    _load().orc_plt_basis(_dp(_v3(n)), _dp(e1), _dp(e2))
    return e1, e2


def plt_point_disk(p, cd, nd, b) -> float:
    return _load().orc_plt_point_disk(_dp(_v3(p)), _dp(_v3(cd)), _dp(_v3(nd)), b)


def plt_rim_near_disk(cc, n_c, a, cd, nd, b, thr):
    """(decision, evaluations) for the rim of the disk (cc, n_c, a) against
    the disk (cd, nd, b) at distance thr."""
    ev = _int(0)
    r = _load().orc_plt_rim_near_disk(_dp(_v3(cc)), _dp(_v3(n_c)), a, _dp(_v3(cd)), _dp(_v3(nd)), b, thr,
                                      ctypes.byref(ev))
    return int(r), int(ev.value)


def plt_collide(dj, ni, nj, a, t) -> int:
    return int(_load().orc_plt_collide(_dp(_v3(dj)), _dp(_v3(ni)), _dp(_v3(nj)), a, t))


def plt_trial(seed, sweep, pid, l, box, c_m, c_r, x0, u0):
    q, u = np.zeros(3), np.zeros(3)
    _load().orc_plt_trial(seed, sweep, pid, l, _dp(_v3(box)), c_m, c_r, _dp(_v3(x0)), _dp(_v3(u0)), _dp(q), _dp(u))
    return q, u


def plt_pairs_brute(box, X, U, a, t, cap: int = 1 << 16):
    X = np.ascontiguousarray(X, dtype=np.float64)
    U = np.ascontiguousarray(U, dtype=np.float64)
    ij = np.zeros((cap, 2), dtype=np.int64)
    cnt = _load().orc_plt_pairs_brute(_dp(_v3(box)), X.shape[0], _dp(X), _dp(U), a, t, ij.ctypes.data_as(P(_i64)),
                                      cap)
    return ij[:min(cnt, cap)].copy(), int(cnt)


def plt_lambda_for_density(box, n, a0, t0, rho) -> float:
    """Scale at which n platelets of base diameter 2 (a0 + t0) reach the
    number density rho = n D^3 / V of Eq. 1 (V the box volume)."""
    V = float(box[0]) * float(box[1]) * float(box[2])
    return (rho * V / n) ** (1.0 / 3.0) / (2.0 * (a0 + t0))


class PlateletSystem:
    """Platelets in the reference: centres X and unit normals U in id order,
    base sizes (a0, t0), scale lambda, target scale, SRM parameters and the
    rotation rate c_r."""

    def __init__(self, box, x, u, a0, t0, lam=1.0, lam_t=None, c_w=0.01, c_m=0.01, c_r=0.0, N_k=10, N_l=10,
                 N_shake=10, seed=1, sweep=0, contact=None, images=False):
        """contact: address of another contact predicate with the signature
        of orc_plt_collide for the sweeps and checks (tests only; None: the
        reference's binary64 decision).  images: periodicity by image
        platelets instead of the minimum image."""
        if not 1 <= N_l < (1 << 16):
            raise ValueError("N_l must be in [1, 65535] (the try index takes 16 counter bits)")
        if not 0.0 <= c_r < 1.0:
            raise ValueError("c_r must be in [0, 1)")
        lib = _load()
        self.box = _v3(box)
        x = np.ascontiguousarray(x, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        self.n = x.size // 3
        self.a0, self.t0 = float(a0), float(t0)
        self._h = lib.orc_plt_create(_dp(self.box), self.n, _dp(x), _dp(u), a0, t0, lam,
                                     lam if lam_t is None else lam_t, c_w, c_m, c_r, N_k, N_l, N_shake, seed, sweep)
        if contact is not None:
            lib.orc_plt_set_contact(self._h, contact)
        lib.orc_plt_set_images(self._h, 1 if images else 0)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.orc_plt_destroy(h)
            self._h = None

    def state(self):
        X, U = np.zeros(3 * self.n), np.zeros(3 * self.n)
        _lib.orc_plt_get(self._h, _dp(X), _dp(U))
        return X.reshape(-1, 3), U.reshape(-1, 3)

    @property
    def lam(self) -> float:
        return _lib.orc_plt_lambda(self._h)

    @property
    def sweep_counter(self) -> int:
        return int(_lib.orc_plt_sweep_counter(self._h))

    def counters(self) -> dict:
        c = np.zeros(5, dtype=np.int64)
        _lib.orc_plt_counters(self._h, c.ctypes.data_as(P(_i64)))
        return dict(iters=int(c[0]), accepted=int(c[1]), shaken=int(c[2]), moves_accepted=int(c[3]),
                    sweeps=int(c[4]))

    def sweep(self) -> int:
        return int(_lib.orc_plt_sweep(self._h))

    def check(self):
        flags = np.zeros(self.n, dtype=np.uint8)
        cnt = _lib.orc_plt_check(self._h, flags.ctypes.data_as(P(ctypes.c_uint8)))
        return int(cnt), flags

    def iterate(self):
        info = np.zeros(3, dtype=np.int64)
        acc = _lib.orc_plt_iterate(self._h, info.ctypes.data_as(P(_i64)))
        return int(acc), dict(k_sweeps=int(info[0]), overlapping=int(info[1]), shake_sweeps=int(info[2]))

    def run(self, max_iters: int = 1 << 40) -> int:
        return int(_lib.orc_plt_run(self._h, max_iters))

    def images_verify(self) -> int:
        return int(_lib.orc_plt_images_verify(self._h))

    def pairs_brute(self):
        X, U = self.state()
        return plt_pairs_brute(self.box, X, U, self.lam * self.a0, self.lam * self.t0)
