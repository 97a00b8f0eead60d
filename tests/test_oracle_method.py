"""Pins of the reference's SRM steps (Algorithms 1 and 3) against closed forms,
invariants, special cases and an independent brute-force sweep."""
import math

import numpy as np
import pytest

import oracle
import srm_inputs
from test_oracle_geometry import brute_pairs_numpy


def _min_image(d, box):
    d = np.where(d > 0.5 * box, d - box, d)
    return np.where(d < -0.5 * box, d + box, d)


def test_phi_closed_form_monodisperse():
    for dim in (2, 3):
        n, R, L = 500, 0.013, 1.3
        X = np.random.default_rng(0).uniform(0, L, size=(n, dim))
        s = oracle.System(dim, [L] * dim, X, np.full(n, R), lam=1.0, c_m=0.001)
        exact = n * math.pi * R**2 / L**2 if dim == 2 else n * 4 / 3 * math.pi * R**3 / L**3
        assert s.phi() == pytest.approx(exact, rel=1e-14)
        for lam in (0.5, 1.7):
            assert s.phi(lam) == pytest.approx(exact * lam**dim, rel=1e-14)
        lt = s.lambda_for_phi(0.3)
        assert s.phi(lt) == pytest.approx(0.3, rel=1e-14)


def test_full_run_disks_1k():
    """The 1000-disk workload reaches 0.50 overlap-free; the number of
    accepted iterations is ceil(ln(lambda_t/lambda_0)/ln(1+c_w)); the scale
    after m accepted iterations is lambda_0 (1+c_w)^m until the cap."""
    w = srm_inputs.disks_1k()
    s = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=w.c_w,
                      c_m=w.c_m, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake, seed=w.seed)
    lam_t = s.lambda_for_phi(w.target_phi)
    assert brute_pairs_numpy(w.x, w.radii, np.array(w.box)).size == 0
    lams, phis = [s.lam], [s.phi()]
    while True:
        acc, info = s.iterate()
        if acc == 2:
            break
        lams.append(s.lam)
        phis.append(s.phi())
        # P stays overlap-free after every iteration
        _, cnt, _ = oracle.pairs_brute(2, w.box, s.x, s.radii())
        assert cnt == 0
    assert np.all(np.diff(phis) >= 0)
    c = s.counters()
    expect = math.ceil(math.log(lam_t) / math.log(1 + w.c_w))
    assert c["accepted"] == expect
    acc_lams = sorted(set(lams))
    for m, lam in enumerate(acc_lams[:-1]):
        assert lam == pytest.approx((1 + w.c_w) ** m, rel=1e-13)
    assert s.lam == lam_t
    assert abs(s.phi() - w.target_phi) < 1e-9
    _, cnt, mg = oracle.pairs_brute(2, w.box, s.x, s.radii())
    assert cnt == 0 and mg > 0


def _overlapping_state(dim, n, seed, swell):
    rng = np.random.default_rng(seed)
    box = np.ones(dim)
    r = np.full(n, (0.25 / n) ** (1 / dim) * 0.5)
    X = srm_inputs.rsa(dim, box, r, seed)
    return box, X, r, swell


@pytest.mark.parametrize("dim", [2, 3])
def test_sweep_invariants(dim):
    box, X, r, swell = _overlapping_state(dim, 600, 9 + dim, 1.35)
    c_m = 0.2 * r[0]
    s = oracle.System(dim, box, X, r, lam=swell, c_m=c_m, N_l=6, seed=4)
    before, _ = s.check()
    assert before > 10
    x0 = s.x
    moved = s.sweep()
    after, _ = s.check()
    # accepted moves never create overlaps: the count cannot grow
    assert after <= before
    d = _min_image(s.x - x0, box)
    step = np.sqrt(np.sum(d * d, axis=1))
    still = step == 0
    # every accepted move has length c_m (up to rounding), the rest did not move
    assert int((~still).sum()) == moved
    np.testing.assert_allclose(step[~still], c_m, rtol=1e-9)


@pytest.mark.parametrize("dim", [2, 3])
def test_single_particle_moves_by_first_try(dim):
    box = np.array([1.0, 0.7, 1.3])[:dim]
    x = np.array([[0.999, 0.01, 0.5][:dim]])
    s = oracle.System(dim, box, x, np.array([0.05]), lam=1.0, c_m=0.03, seed=99)
    for k in range(20):
        before = s.x[0].copy()
        u, _ = oracle.unit_dir(99, k, 0, 0, dim)
        assert s.sweep() == 1
        expect = np.array([oracle.wrap(before[a] + 0.03 * u[a], box[a]) for a in range(dim)])
        np.testing.assert_array_equal(s.x[0], expect)


def test_jammed_lattice_does_not_move():
    """A square lattice of disks 1e-9 short of contact: every trial move of
    length c_m brings some neighbour within contact, so nothing moves."""
    m = 12
    a = 1.0 / m
    g = (np.arange(m) + 0.5) * a
    X = np.array([(x, y) for y in g for x in g])
    R = 0.5 * a * (1 - 1e-9)
    s = oracle.System(2, [1.0, 1.0], X, np.full(m * m, R), lam=1.0, c_m=0.05 * a, N_l=10)
    assert s.check()[0] == 0
    x0 = s.x
    assert s.sweep() == 0
    np.testing.assert_array_equal(s.x, x0)


def canonical_order(X, box, lam, rmax, c_m):
    """Colour -> cell -> id order of the canonical sweep, restated from the
    reading of Algorithm 3's particle order (not from the reference's code)."""
    dim = X.shape[1]
    n, w = oracle.grid(dim, box, lam, rmax, c_m)
    c = np.floor(X / w).astype(np.int64) % n
    col = np.zeros(len(X), dtype=np.int64)
    lin = np.zeros(len(X), dtype=np.int64)
    mul = 1
    for a in range(dim):
        col += (c[:, a] % 3) * 3**a
        lin += c[:, a] * mul
        mul *= int(n[a])
    return np.lexsort((np.arange(len(X)), lin, col))


def brute_sweep(X, r, lam, box, c_m, N_l, seed, sweep, order):
    """Algorithm 3 with an O(N) collision test per trial (no cell list)."""
    X = X.copy()
    dim = X.shape[1]
    R = lam * r
    for pid in order:
        q_old = X[pid].copy()
        for l in range(N_l):
            u, _ = oracle.unit_dir(seed, sweep, int(pid), l, dim)
            q = q_old + c_m * u[:dim]
            q = np.where(q < 0, q + box, q)
            q = np.where(q >= box, q - box, q)
            d = _min_image(q - X, box)
            ss = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
            if dim == 3:
                ss = ss + d[:, 2] * d[:, 2]
            S = np.sqrt(ss)
            S[pid] = np.inf
            if not np.any(S <= R[pid] + R):
                X[pid] = q
                break
    return X


@pytest.mark.parametrize("dim,literal", [(2, False), (3, False), (2, True), (3, True)])
def test_sweep_equals_brute_force(dim, literal):
    box, X, r, swell = _overlapping_state(dim, 300, 21 + dim, 1.25)
    box = box * np.array([1.0, 1.1, 0.9])[:dim]
    c_m = 0.3 * r[0]
    s = oracle.System(dim, box, X, r, lam=swell, c_m=c_m, N_l=5, seed=17, sweep=3,
                      literal=literal)
    order = np.arange(len(X)) if literal else canonical_order(X, box, swell, r.max(), c_m)
    expect = brute_sweep(X, r, swell, box, c_m, 5, 17, 3, order)
    s.sweep()
    np.testing.assert_array_equal(s.x, expect)
    # a second sweep from the new state, with the counter advanced
    order2 = np.arange(len(X)) if literal else canonical_order(expect, box, swell, r.max(), c_m)
    expect2 = brute_sweep(expect, r, swell, box, c_m, 5, 17, 4, order2)
    s.sweep()
    np.testing.assert_array_equal(s.x, expect2)


def test_shake_path():
    """A swelling step too large to resolve in N_k sweeps is discarded: P keeps
    its scale, is shaken N_shake times and stays overlap-free."""
    box, X, r, _ = _overlapping_state(2, 400, 31, 1.0)
    s = oracle.System(2, box, X, r, lam=1.0, lam_t=10.0, c_w=0.9, c_m=0.02 * r[0], N_k=2,
                      N_l=2, N_shake=3, seed=8)
    x0 = s.x
    acc, info = s.iterate()
    assert acc == 0 and info["shake_sweeps"] == 3 and info["overlapping"] > 0
    assert s.lam == 1.0
    assert s.sweep_counter == 2 + 3
    assert oracle.pairs_brute(2, box, s.x, s.radii())[1] == 0
    assert not np.array_equal(s.x, x0)


@pytest.mark.parametrize("literal", [False, True])
def test_literal_and_canonical_reach_target(literal):
    w = srm_inputs.disks_1k(seed=4, n=400)
    s = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=0.55, c_w=0.02,
                      c_m=w.c_m, seed=4, literal=literal)
    s.run()
    assert abs(s.phi() - 0.55) < 1e-9
    assert oracle.pairs_brute(2, w.box, s.x, s.radii())[1] == 0
