"""Pins of the reference's geometry: periodic wrap (Algorithm 4), the grid
rule (Algorithm 1, Algorithm 2), and the cell-list overlap search
(Algorithms 5 and 6) against O(N^2) brute force and periodic-image
invariance."""
import numpy as np
import pytest

import oracle


def test_wrap_special_cases():
    L = 1.0
    assert oracle.wrap(0.25, L) == 0.25
    assert oracle.wrap(-0.25, L) == 0.75
    assert oracle.wrap(1.25, L) == 0.25
    assert oracle.wrap(L, L) == 0.0
    assert oracle.wrap(0.0, L) == 0.0
    # -tiny + L rounds to L; the ">= L" test that follows maps it to 0
    tiny = 1e-20
    assert -tiny + L == L
    assert oracle.wrap(-tiny, L) == 0.0
    # just below L stays
    below = np.nextafter(L, 0.0)
    assert oracle.wrap(below, L) == below
    # a box that is not a power of two
    L3 = 0.3
    assert oracle.wrap(-0.1, L3) == -0.1 + L3
    assert 0.0 <= oracle.wrap(-1e-18, L3) < L3


@pytest.mark.parametrize("dim", [2, 3])
def test_grid_rule(dim):
    rng = np.random.default_rng(3)
    for _ in range(200):
        box = rng.uniform(0.5, 3.0, size=dim)
        rmax = rng.uniform(1e-3, 0.05)
        lam = rng.uniform(0.5, 2.0)
        c_m = rng.uniform(0.0, 0.5) * lam * rmax
        n, w = oracle.grid(dim, box, lam, rmax, c_m)
        cs = 2.5 * lam * rmax + c_m
        assert np.all(n % 3 == 0) and np.all(n >= 3)
        for a in range(dim):
            if box[a] >= 3 * cs:
                assert w[a] >= cs * (1 - 1e-15)
                # the largest multiple of 3 with w >= cellSize
                assert box[a] / (n[a] + 3) < cs
            assert w[a] == box[a] / n[a]


def brute_pairs_numpy(X, R, box):
    """O(N^2) pair list, written with numpy independently of the reference."""
    n, dim = X.shape
    out = []
    for i in range(n):
        d = X[i] - X[i + 1:]
        for a in range(dim):
            da = d[:, a]
            da = np.where(da > 0.5 * box[a], da - box[a], da)
            da = np.where(da < -0.5 * box[a], da + box[a], da)
            d[:, a] = da
        ss = d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]
        if dim == 3:
            ss = ss + d[:, 2] * d[:, 2]
        hit = np.nonzero(np.sqrt(ss) <= R[i] + R[i + 1:])[0]
        out.extend((i, i + 1 + j) for j in hit)
    return np.array(out, dtype=np.int64).reshape(-1, 2)


def _random_state(rng, dim, n, box, r_lo, r_hi):
    X = rng.uniform(0, 1, size=(n, dim)) * np.asarray(box)[:dim]
    r = rng.uniform(r_lo, r_hi, size=n)
    return X, r


@pytest.mark.parametrize("dim,n", [(2, 400), (3, 400), (2, 1500), (3, 1200)])
def test_cell_pairs_equal_brute_force(dim, n):
    rng = np.random.default_rng(dim * 100 + n)
    box = rng.uniform(0.8, 1.5, size=dim)
    X, r = _random_state(rng, dim, n, box, 0.005, 0.04)
    s = oracle.System(dim, box, X, r, lam=1.0, c_m=0.01)
    p = s.pairs()
    q = brute_pairs_numpy(X, r, box)
    assert len(q) > 20
    np.testing.assert_array_equal(p, q)
    ref, cnt, _ = oracle.pairs_brute(dim, box, X, r)
    np.testing.assert_array_equal(ref, q)
    # Algorithm 6 with a full count: the particles that appear in some pair
    cnt_check, flags = s.check()
    involved = np.zeros(n, dtype=np.uint8)
    involved[q.ravel()] = 1
    np.testing.assert_array_equal(flags, involved)
    assert cnt_check == int(involved.sum())
    # cell-list certification agrees on the count
    c, mg = oracle.certify(dim, box, X, r)
    assert c == len(q) and mg <= 0


@pytest.mark.parametrize("dim", [2, 3])
def test_adversarial_positions(dim):
    """Particles on cell faces, at L - eps, at 0, on the grid with n = 3 and 6."""
    rng = np.random.default_rng(77 + dim)
    box = np.ones(dim)
    for rad, c_m in [(0.1, 0.02), (0.05, 0.01), (0.03, 0.004)]:
        n, w = oracle.grid(dim, box, 1.0, rad, c_m)
        faces = np.concatenate([np.arange(n[0] + 1) * w[0], [1 - 1e-16, 1e-300, 0.5]])
        pts = []
        for _ in range(300):
            p = [rng.choice(faces) if rng.random() < 0.6 else rng.random() for _ in range(dim)]
            pts.append([min(v, np.nextafter(1.0, 0)) for v in p])
        X = np.array(pts)
        r = np.full(len(X), rad) * rng.uniform(0.5, 1.0, size=len(X))
        s = oracle.System(dim, box, X, r, lam=1.0, c_m=c_m)
        np.testing.assert_array_equal(s.pairs(), brute_pairs_numpy(X, r, box))


@pytest.mark.parametrize("dim", [2, 3])
def test_periodic_image_invariance(dim):
    rng = np.random.default_rng(5 + dim)
    box = np.array([1.0, 0.5, 2.0])[:dim]
    X, r = _random_state(rng, dim, 800, box, 0.01, 0.03)
    base = oracle.System(dim, box, X, r, lam=1.0, c_m=0.005).pairs()
    assert len(base) > 10
    # a shift by a multiple of the box is exact and leaves every pair in place
    for a in range(dim):
        for sgn in (-1, 1):
            Y = X.copy()
            Y[:, a] = Y[:, a] + sgn * box[a]
            Y[:, a] = np.where(Y[:, a] < 0, Y[:, a] + box[a], Y[:, a])
            Y[:, a] = np.where(Y[:, a] >= box[a], Y[:, a] - box[a], Y[:, a])
            np.testing.assert_array_equal(
                oracle.System(dim, box, Y, r, lam=1.0, c_m=0.005).pairs(), base)
    # a shift by a random vector mod L: compare with brute force on the
    # shifted state (rounding may move a pair across the contact threshold)
    shift = rng.uniform(0, 1, size=dim) * box
    Y = np.mod(X + shift, box)
    Y = np.where(Y >= box, 0.0, Y)
    got = oracle.System(dim, box, Y, r, lam=1.0, c_m=0.005).pairs()
    np.testing.assert_array_equal(got, brute_pairs_numpy(Y, r, box))
    sym = set(map(tuple, got)) ^ set(map(tuple, base))
    assert len(sym) <= 2
