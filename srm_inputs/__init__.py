"""Seeded synthetic inputs for SRM runs (radii and RSA starting configurations).

This module holds no step of the SRM method.  It builds the starting state
that the paper's main loop takes as given (Section 2: non-overlapping
particles at a low initial volume fraction f0 placed by random sequential
addition; Algorithm 1) and the workload recipes used by the tests and
the benchmark.  The FP64 reference and the CUDA library are both fed from
here, so that they receive identical inputs; neither is imported by it.

Workload recipes (sizes and distributions of the paper's benchmarks, Section
3.1: RSA at f0 = 0.1, then swelling to 0.5 in 2D and 0.4 in 3D):

* ``disks_1k``     2D, N=1000, unit square, monodisperse, target 0.50.
* ``spheres_100k`` 3D, N=1e5, unit cube, monodisperse, target 0.45.
* ``poly_1m``      3D, N=1e6, log-normal radii (mean 1, sd 0.2, truncated to
  [0.5, 2]), 200 Gaussian clusters with sigma = 5 mean radii, target 0.40.
* ``spheres_10m``  3D, N=1e7, unit cube, monodisperse, target 0.30.
* ``ensemble``     many independent RVEs: half disks, half spheres, N
  log-uniform in [1e3, 1e5], targets uniform in [0.30, 0.55].

Radii are returned at the starting scale (the radii of the RSA placement), so
that the starting scale factor is 1; the target scale follows from the target
fraction.  The migration step c_m is 0.1 of the mean radius at the target.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libsrm_inputs.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into a shared library (plain gcc, no CUDA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i64, u64 = ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
            lib.inp_radii_lognormal.argtypes = [i64, d, d, d, d, u64, P(d)]
            lib.inp_radii_lognormal.restype = ctypes.c_int
            lib.inp_rsa.argtypes = [ctypes.c_int, P(d), i64, P(d), u64, ctypes.c_int, i64, d, i64,
                                    P(d)]
            lib.inp_rsa.restype = ctypes.c_int
            lib.inp_uniforms.argtypes = [u64, u64, i64, P(d)]
            lib.inp_uniforms.restype = None
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def radii_lognormal(n: int, mean: float, sd: float, lo: float, hi: float, seed: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    if _load().inp_radii_lognormal(n, mean, sd, lo, hi, seed, _dp(out)) != 0:
        raise RuntimeError("log-normal radii: truncation window too narrow")
    return out


def rsa(dim: int, box, radii: np.ndarray, seed: int, clusters: int = 0, sigma: float = 0.0,
        max_attempts: int = 10_000_000) -> np.ndarray:
    """Non-overlapping positions (n, dim) by random sequential addition."""
    radii = np.ascontiguousarray(radii, dtype=np.float64)
    L = np.zeros(3)
    L[:dim] = box[:dim]
    X = np.zeros((radii.size, dim), dtype=np.float64)
    rc = _load().inp_rsa(dim, _dp(L), radii.size, _dp(radii), seed, 1 if clusters > 0 else 0,
                         clusters, sigma, max_attempts, _dp(X))
    if rc != 0:
        raise RuntimeError("RSA could not place every particle")
    return X


def uniforms(seed: int, tag: int, n: int) -> np.ndarray:
    out = np.empty(n, dtype=np.float64)
    _load().inp_uniforms(seed, tag, n, _dp(out))
    return out


@dataclass
class Workload:
    """One RVE: box, dimension, starting radii and positions, and parameters."""
    name: str
    dim: int
    box: tuple
    radii: np.ndarray          # radii at the start (scale factor 1)
    x: np.ndarray              # (n, dim) starting positions, non-overlapping
    target_phi: float
    seed: int
    c_w: float = 0.01
    c_m: float = 0.0
    N_k: int = 10
    N_l: int = 10
    N_shake: int = 10
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.radii.size)


def _mono(name, dim, n, phi_t, f0, seed, box=1.0):
    vol = box ** dim
    if dim == 2:
        r_t = math.sqrt(phi_t * vol / (n * math.pi))
    else:
        r_t = (phi_t * vol * 3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r0 = r_t * (f0 / phi_t) ** (1.0 / dim)
    radii = np.full(n, r0)
    x = rsa(dim, (box,) * dim, radii, seed)
    return Workload(name, dim, (box,) * dim, radii, x, phi_t, seed, c_m=0.1 * r_t,
                    extra={"r_target": r_t, "f0": f0})


def disks_1k(seed: int = 1, n: int = 1000, phi_t: float = 0.50, f0: float = 0.1) -> Workload:
    return _mono("disks_1k", 2, n, phi_t, f0, seed)


def spheres_100k(seed: int = 2, n: int = 100_000, phi_t: float = 0.45, f0: float = 0.1) -> Workload:
    return _mono("spheres_100k", 3, n, phi_t, f0, seed)


def spheres_10m(seed: int = 5, n: int = 10_000_000, phi_t: float = 0.30, f0: float = 0.1) -> Workload:
    return _mono("spheres_10m", 3, n, phi_t, f0, seed)


def poly_1m(seed: int = 3, n: int = 1_000_000, phi_t: float = 0.40, f0: float = 0.1,
            clusters: int = 200, sigma_in_radii: float = 5.0) -> Workload:
    """Polydisperse clustered spheres: radii at the target drawn log-normal
    (mean 1, sd 0.2, truncated to [0.5, 2]); the box is sized so that these
    radii fill phi_t; the start is RSA at f0 with proposals from 200 Gaussian
    clusters of standard deviation 5 mean radii."""
    r_t = radii_lognormal(n, 1.0, 0.2, 0.5, 2.0, seed)
    vol_t = float(np.sum(4.0 / 3.0 * math.pi * r_t ** 3))
    box = (vol_t / phi_t) ** (1.0 / 3.0)
    radii = r_t * (f0 / phi_t) ** (1.0 / 3.0)
    mean_r = float(np.mean(r_t))
    x = rsa(3, (box,) * 3, radii, seed, clusters=clusters, sigma=sigma_in_radii * mean_r)
    return Workload("poly_1m", 3, (box,) * 3, radii, x, phi_t, seed, c_m=0.1 * mean_r,
                    extra={"r_target_mean": mean_r, "f0": f0, "clusters": clusters})


def ensemble(count: int = 256, seed0: int = 0, n_lo: float = 1e3, n_hi: float = 1e5,
             phi_lo: float = 0.30, phi_hi: float = 0.55, f0: float = 0.1) -> list:
    """Independent RVEs: the first half disks, the second half spheres; RVE i
    draws its size log-uniform in [n_lo, n_hi] and its target uniform in
    [phi_lo, phi_hi] from the input stream of seed i, and runs with seed i."""
    return [ensemble_member(i, count, seed0, n_lo, n_hi, phi_lo, phi_hi, f0) for i in range(count)]


def ensemble_member(i: int, count: int = 256, seed0: int = 0, n_lo: float = 1e3, n_hi: float = 1e5,
                    phi_lo: float = 0.30, phi_hi: float = 0.55, f0: float = 0.1) -> Workload:
    """RVE i of ensemble(count, seed0, ...)."""
    u = uniforms(seed0 + i, 0x4D455441, 2)  # "META"
    n = int(math.floor(n_lo * (n_hi / n_lo) ** u[0]))
    phi_t = phi_lo + (phi_hi - phi_lo) * u[1]
    dim = 2 if i < count // 2 else 3
    return _mono(f"ensemble[{i}]", dim, n, phi_t, f0, seed0 + i)


@dataclass
class PlateletWorkload:
    """Thin platelets (spherodisks, Section 3.3) in a box: base sizes (a0,
    t0) of the target (scale 1), starting scale lambda0, centres x and unit
    normals u (n x 3) of a collision-free start, and SRM parameters."""
    name: str
    box: tuple
    a0: float
    t0: float
    lambda0: float
    x: np.ndarray
    u: np.ndarray
    rho_t: float
    seed: int
    c_w: float
    c_m: float
    c_r: float
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def platelets(seed: int = 7, n: int = 20_000, aspect: float = 100.0, rho_t: float = 5.0, f0: float = 0.1,
              c_w: float = 0.01, c_m_rel: float = 0.02, c_r: float = 0.02, box: float = 1.0) -> PlateletWorkload:
    """n identical platelets of aspect ratio D / (2 t) = aspect in a cubic box,
    sized so that the target is the number density rho_t of Eq. 1 (rho =
    n D^3 / V) at scale 1.  Start: random sequential addition of the bounding
    spheres (radius a + t) at volume fraction f0 -- bounding spheres that do
    not overlap leave the platelets apart -- with uniform random normals.
    Default parameters are those of a "house of cards" run: swelling of 1% per
    iteration against short migration steps (c_m = c_m_rel D, twice the
    thickness at aspect 100) and small turns (c_r)."""
    V = box ** 3
    D = (rho_t * V / n) ** (1.0 / 3.0)
    t0 = D / (2.0 * aspect)
    a0 = D / 2.0 - t0
    Rb = a0 + t0
    lam0 = (f0 * V / (n * 4.0 / 3.0 * math.pi)) ** (1.0 / 3.0) / Rb
    x = rsa(3, (box,) * 3, np.full(n, lam0 * Rb), seed)
    w = uniforms(seed, 0x4E524D4C, 2 * n)  # "NRML"
    z = 2.0 * w[:n] - 1.0
    ph = 2.0 * math.pi * w[n:]
    s = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    u = np.stack([s * np.cos(ph), s * np.sin(ph), z], axis=1)
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    return PlateletWorkload("platelets", (box,) * 3, a0, t0, lam0, x, u, rho_t, seed, c_w, c_m_rel * D, c_r,
                            extra={"aspect": aspect, "D": D, "f0": f0})


RECIPES = {
    "disks_1k": disks_1k,
    "spheres_100k": spheres_100k,
    "poly_1m": poly_1m,
    "spheres_10m": spheres_10m,
}
