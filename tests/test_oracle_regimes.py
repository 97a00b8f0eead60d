"""The reference reproduces the qualitative result of Section 3.2 (Fig. 5):
at the same volume fraction, fast swelling with migration just long enough
to clear the overlaps of one swell step leaves clustered configurations,
whose local volume fractions (particle area over Voronoi-cell area) spread
clearly more than after slow swelling with long migration.  2000 disks to
0.5 from an RSA start at 0.1, two seeds per regime; both end certified.
Also the dense limits that Section 2 states."""
import math

import numpy as np
import pytest

import oracle
import srm_inputs


def lvf_spread(c_w, c_m_rel, seed, n=2000, phi=0.5):
    r_t = math.sqrt(phi / (n * math.pi))
    r0 = r_t * math.sqrt(0.1 / phi)
    x = srm_inputs.rsa(2, (1.0, 1.0), np.full(n, r0), seed)
    s = oracle.System(2, (1.0, 1.0), x, np.full(n, r0), lam=1.0, target_phi=phi, c_w=c_w, c_m=c_m_rel * r_t,
                      seed=seed)
    s.run()
    X, R = s.x, s.radii()
    assert abs(s.phi() - phi) < 1e-12
    assert oracle.certify(2, (1.0, 1.0), X, R)[0] == 0
    _, lvf = oracle.voronoi_lvf(2, (1.0, 1.0), X, R, (200, 200))
    _, _, gap = oracle.nn(2, (1.0, 1.0), X, R)
    return float(np.std(lvf)), float(np.mean(gap)) / (2.0 * float(R[0]))


def test_clustered_regime_spreads_local_volume_fraction():
    """LVF spread (Fig. 5) and the nearest-neighbour gaps (Fig. 4d: the
    clustered configuration has its neighbours closer)."""
    eq = np.mean([lvf_spread(0.002, 0.5, s) for s in (1, 2)], axis=0)
    cl = np.mean([lvf_spread(0.01, 0.03, s) for s in (1, 2)], axis=0)
    assert cl[0] > 1.4 * eq[0], (cl, eq)
    assert cl[1] < 0.7 * eq[1], (cl, eq)


def dense_run(dim, n, phi, seed, c_w, c_m_rel, cap_s=120.0):
    import time
    r_t = math.sqrt(phi / (n * math.pi)) if dim == 2 else (phi * 3.0 / (4.0 * math.pi * n)) ** (1.0 / 3.0)
    r0 = r_t * (0.1 / phi) ** (1.0 / dim)
    box = (1.0,) * dim
    x = srm_inputs.rsa(dim, box, np.full(n, r0), seed)
    s = oracle.System(dim, box, x, np.full(n, r0), lam=1.0, target_phi=phi, c_w=c_w, c_m=c_m_rel * r_t, seed=seed)
    t0 = time.perf_counter()
    while s.lam < s.lambda_for_phi(phi) and time.perf_counter() - t0 < cap_s:
        s.run(200)
    return s, box


def test_dense_limits():
    """Section 2: with small swelling and migration rates SRM goes past the
    random-close-packing fraction of monodisperse disks (0.82) and reaches
    about 0.60 for monodisperse spheres.  1000 disks to 0.84 and 1000 spheres
    to 0.60, certified."""
    for dim, phi, seed in ((2, 0.84, 5), (3, 0.60, 3)):
        s, box = dense_run(dim, 1000, phi, seed, 0.0005 if dim == 2 else 0.001, 0.05)
        assert s.phi() == pytest.approx(phi, abs=1e-12), (dim, s.phi())
        assert oracle.certify(dim, box, s.x, s.radii())[0] == 0
