"""Pins of the reference's image-particle periodicity (Section 2: images are
added or removed as particles cross the boundary, the alternative to the
minimum image of Alg 5).

* Colliding pairs equal a brute force over explicit periodic copies built
  here (every particle shifted by every s in {-1,0,1}^d, plain differences
  q - (x + s L) in binary64, the same operations): exactly, in 2D and 3D,
  with particles crowded against the faces, edges and corners.
* Decisions equal the minimum-image ones: pair sets, and whole sweeps and
  iterations of Algorithm 1, bit for bit (the two arithmetics round the
  periodic difference differently, so only a pair within rounding of
  contact could decide otherwise).
* The entries kept move by move during a sweep equal a rebuild from the
  final positions (images added and removed at every crossing), and their
  number matches the particles in boundary cells.
"""
import itertools

import numpy as np
import pytest

import oracle
import srm_inputs


def brute_images(dim, box, X, R):
    """Pairs i < j colliding with some periodic copy x_j + s L of j."""
    L = np.asarray(box, dtype=np.float64)
    n = len(R)
    out = set()
    for s in itertools.product((-1, 0, 1), repeat=dim):
        Y = X + np.asarray(s, dtype=np.float64) * L  # x_j + s L, one rounding per axis
        for i in range(n):
            d = X[i] - Y  # q - y
            ss = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
            if dim == 3:
                ss = ss + d[:, 2] * d[:, 2]
            hit = np.nonzero(np.sqrt(ss) <= R[i] + R)[0]
            out.update((i, int(j)) for j in hit if j > i)
    return sorted(out)


def crowded(dim, n, seed):
    """Random polydisperse particles, a third of them pressed against the
    faces (within one radius of 0 or L on some axes)."""
    rng = np.random.default_rng(seed)
    box = (1.0, 0.9, 1.1)[:dim]
    r = rng.uniform(0.02, 0.05, n) if dim == 3 else rng.uniform(0.01, 0.03, n)
    x = rng.uniform(0, 1, (n, dim)) * np.asarray(box)
    k = n // 3
    for a in range(dim):
        side = rng.integers(0, 2, k).astype(bool)
        x[:k, a] = np.where(side, rng.uniform(0, 0.05, k), np.asarray(box)[a] - rng.uniform(1e-9, 0.05, k))
    return box, x, r


@pytest.mark.parametrize("dim,n,seed", [(2, 900, 1), (3, 700, 2), (3, 400, 3)])
def test_pairs_equal_brute_force_over_explicit_copies(dim, n, seed):
    box, x, r = crowded(dim, n, seed)
    s = oracle.System(dim, box, x, r, images=True)
    got = [tuple(p) for p in s.pairs().tolist()]
    ref = brute_images(dim, box, x, r)
    assert len(ref) > 20
    assert got == ref
    assert s.images_count() > 0


@pytest.mark.parametrize("dim,n,seed", [(2, 900, 4), (3, 700, 5)])
def test_pairs_equal_minimum_image(dim, n, seed):
    box, x, r = crowded(dim, n, seed)
    a = oracle.System(dim, box, x, r)
    b = oracle.System(dim, box, x, r, images=True)
    np.testing.assert_array_equal(a.pairs(), b.pairs())
    np.testing.assert_array_equal(a.check()[1], b.check()[1])


@pytest.mark.parametrize("maker", [lambda: srm_inputs.disks_1k(seed=6, n=600),
                                   lambda: srm_inputs._mono("s3", 3, 900, 0.40, 0.1, 7)])
def test_runs_equal_minimum_image_and_images_stay_consistent(maker):
    w = maker()
    args = dict(lam=1.0, target_phi=w.target_phi, c_w=0.04, c_m=w.c_m, seed=w.seed)
    a = oracle.System(w.dim, w.box, w.x, w.radii, **args)
    b = oracle.System(w.dim, w.box, w.x, w.radii, images=True, **args)
    for _ in range(6):
        ra, ia = a.iterate()
        rb, ib = b.iterate()
        assert (ra, ia) == (rb, ib)
        np.testing.assert_array_equal(a.x, b.x)
    # sweeps of P at its scale: the same moves, and the entries kept move by
    # move equal a rebuild from the final positions
    for _ in range(3):
        mb = b.sweep()
        assert a.sweep() == mb > 0
        assert b.images_verify() == 0
        np.testing.assert_array_equal(a.x, b.x)
    assert b.run() >= 0 and a.run() >= 0
    np.testing.assert_array_equal(a.x, b.x)
    assert b.counters() == a.counters()
    assert oracle.pairs_brute(w.dim, w.box, b.x, b.radii())[1] == 0


def test_image_count_matches_boundary_cells():
    """Images exist exactly for particles of the first and last cell layer
    along an axis: one per boundary axis, three more for an edge in 2D."""
    box = (1.0, 1.0)
    r = np.full(4, 0.01)
    x = np.array([[0.001, 0.5], [0.5, 0.999], [0.001, 0.999], [0.5, 0.5]])
    s = oracle.System(2, box, x, r, images=True)
    s.check()
    assert s.images_count() == 1 + 1 + 3


def test_platelet_sweeps_and_checks_equal_minimum_image():
    """Platelets (Section 3.3) with image platelets: sweeps with rotation
    and Alg 6 flags equal the minimum-image ones bit for bit, on platelets
    crowded against the faces; the entries stay consistent move by move."""
    from test_oracle_platelet import rand_units
    rng = np.random.default_rng(8)
    n = 400
    box = (1.0, 1.0, 1.0)
    x = rng.uniform(0, 1, (n, 3))
    x[:n // 3, 0] = rng.uniform(0, 0.03, n // 3)
    u = rand_units(rng, n)
    a0, t0 = 0.03, 0.003
    args = dict(lam=1.0, lam_t=1.0, c_m=0.01, c_r=0.1, N_l=4, seed=3)
    a = oracle.PlateletSystem(box, x, u, a0, t0, **args)
    b = oracle.PlateletSystem(box, x, u, a0, t0, images=True, **args)
    fa, fb = a.check()[1], b.check()[1]
    assert fa.sum() > 10
    np.testing.assert_array_equal(fa, fb)
    for _ in range(3):
        assert a.sweep() == b.sweep()
        assert b.images_verify() == 0
        xa, ua = a.state()
        xb, ub = b.state()
        np.testing.assert_array_equal(xa, xb)
        np.testing.assert_array_equal(ua, ub)
