"""Pins of the platelet reference (spherodisks, Section 3.3).

The contact test decides "disk-to-disk distance <= t_i + t_j" in binary64;
a pair within 2e-12 a of touching that its rim search cannot resolve counts
as contact.

* The contact decision against the distance between two disks found by brute
  force (dense point clouds of both disks, nearest pair by a KD-tree, refined
  by a local optimiser): the threshold at which the decision flips must lie
  between the brute-force lower and upper bounds.
* Closed-form configurations: coplanar disks, stacked parallel disks, a disk
  standing on another (T), two disks meeting edge to edge at a right angle.
* Invariances: swapping the two platelets, a rigid rotation of the pair.
* Point-to-disk distance against a sampled disk.
* The sweep against a brute-force sweep written here (every platelet tested,
  no cell list, order recomputed from the reading), a lone platelet's move,
  Alg 6 against brute-force pairs, and whole iterations (collision-free P,
  scale progression, the number density of Eq. 1).
"""
import math

import numpy as np
import pytest

import oracle

spatial = pytest.importorskip("scipy.spatial")
optimize = pytest.importorskip("scipy.optimize")

CLEAR = 1e-9  # a gap this much beyond 2 t (times a) is clear of the rim search's resolution and of rounding


def unit(v):
    v = np.asarray(v, dtype=np.float64)
    return v / np.linalg.norm(v)


def rand_units(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def disk_basis(n):
    """An orthonormal in-plane basis, built here independently of the oracle."""
    a = np.array([1.0, 0.0, 0.0]) if abs(n[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = unit(np.cross(n, a))
    return e1, np.cross(n, e1)


def disk_cloud(c, n, a, nr=50, nt=400):
    e1, e2 = disk_basis(n)
    r = np.linspace(a / nr, a, nr)
    th = np.linspace(0.0, 2 * math.pi, nt, endpoint=False)
    R, T = np.meshgrid(r, th, indexing="ij")
    pts = c + (R * np.cos(T))[..., None] * e1 + (R * np.sin(T))[..., None] * e2
    err = a / nr + 0.5 * a * (2 * math.pi / nt)  # farthest disk point from a sample
    return np.vstack([np.asarray(c, dtype=np.float64)[None], pts.reshape(-1, 3)]), err


def brute_distance(ci, ni, cj, nj, a):
    """(lower, upper) bounds of the distance between two disks of radius a."""
    # a coarse pass bounds the answer from above, so that the fine KD-tree
    # query only has to search within that bound
    Pc, _ = disk_cloud(ci, ni, a, 10, 60)
    Qc, _ = disk_cloud(cj, nj, a, 10, 60)
    M = np.linalg.norm(Pc[:, None, :] - Qc[None, :, :], axis=2)
    ic, jc = np.unravel_index(int(np.argmin(M)), M.shape)
    bound = float(M[ic, jc])
    P, err = disk_cloud(ci, ni, a)
    Q, _ = disk_cloud(cj, nj, a)
    d, k = spatial.cKDTree(Q).query(P, distance_upper_bound=bound * (1 + 1e-9) + 1e-12)
    i0 = int(np.argmin(d))
    if np.isinf(d[i0]):  # no fine pair within the coarse bound: fine minimum >= bound
        coarse, p0, q0 = bound, Pc[ic], Qc[jc]
    else:
        coarse, p0, q0 = float(d[i0]), P[i0], Q[k[i0]]
    ei1, ei2 = disk_basis(ni)
    ej1, ej2 = disk_basis(nj)

    def pt(c, e1, e2, r, t):
        r = min(max(r, 0.0), a)
        return c + r * math.cos(t) * e1 + r * math.sin(t) * e2

    def f(z):
        return float(np.linalg.norm(pt(ci, ei1, ei2, z[0], z[1]) - pt(cj, ej1, ej2, z[2], z[3])))

    def polar(p, c, e1, e2):
        v = p - c
        x, y = float(v @ e1), float(v @ e2)
        return [math.hypot(x, y), math.atan2(y, x)]

    z0 = polar(p0, ci, ei1, ei2) + polar(q0, cj, ej1, ej2)
    res = optimize.minimize(f, z0, method="Nelder-Mead", options=dict(xatol=1e-11, fatol=1e-13, maxiter=1500))
    upper = min(coarse, f(res.x))
    return coarse - 2 * err, upper


def flip_threshold(dj, ni, nj, a, lo=0.0, hi=None):
    """Smallest thr = 2 t at which the decision says "collision", by
    bisection on t (the decision is monotone in the threshold)."""
    hi = hi if hi is not None else 4 * a
    tl, th = lo / 2, hi / 2
    assert oracle.plt_collide(dj, ni, nj, a, th) == 1
    for _ in range(60):
        tm = 0.5 * (tl + th)
        if oracle.plt_collide(dj, ni, nj, a, tm):
            th = tm
        else:
            tl = tm
    return 2 * th


def test_point_disk_against_sampled_disk():
    rng = np.random.default_rng(1)
    for _ in range(40):
        cd = rng.normal(size=3)
        nd = unit(rng.normal(size=3))
        b = rng.uniform(0.2, 1.5)
        p = cd + rng.normal(size=3) * 1.5
        P, err = disk_cloud(cd, nd, b, 200, 1600)
        ref = float(np.min(np.linalg.norm(P - p, axis=1)))
        d = oracle.plt_point_disk(p, cd, nd, b)
        assert ref - err - 1e-12 <= d <= ref + 1e-12


def test_point_disk_closed_forms():
    nd = np.array([0.0, 0.0, 1.0])
    assert oracle.plt_point_disk([0.3, -0.2, 0.7], [0, 0, 0], nd, 1.0) == pytest.approx(0.7, abs=1e-15)
    assert oracle.plt_point_disk([3.0, 4.0, 0.0], [0, 0, 0], nd, 1.0) == pytest.approx(4.0, abs=1e-15)
    assert oracle.plt_point_disk([0.0, 2.0, -2.0], [0, 0, 0], nd, 1.0) == pytest.approx(math.sqrt(5.0), abs=1e-15)


def test_basis_orthonormal():
    rng = np.random.default_rng(2)
    for n in list(rand_units(rng, 200)) + [np.eye(3)[k] for k in range(3)]:
        e1, e2 = oracle.plt_basis(n)
        M = np.stack([e1, e2, n])
        np.testing.assert_allclose(M @ M.T, np.eye(3), atol=1e-15)


@pytest.mark.parametrize("seed", [3, 4])
def test_decision_threshold_equals_brute_force_distance(seed):
    rng = np.random.default_rng(seed)
    a = 1.0
    checked = 0
    for _ in range(20):
        ni, nj = rand_units(rng, 2)
        dj = rng.normal(size=3)
        dj *= rng.uniform(0.8, 2.2) / np.linalg.norm(dj)
        lo, up = brute_distance(np.zeros(3), ni, dj, nj, a)
        if up <= 1e-9:
            assert oracle.plt_collide(dj, ni, nj, a, 1e-6) == 1
            continue
        d = flip_threshold(dj, ni, nj, a)
        # the decision may count a near-contact it cannot resolve as contact,
        # never a clear gap: the flip lies in [lower bound - resolution, upper]
        assert max(lo, 0.0) - 1e-9 <= d <= up + 1e-9, (d, lo, up)
        checked += 1
    assert checked >= 12


@pytest.mark.parametrize("aspect", [5.0, 100.0])
def test_decision_on_near_contacts_matches_brute_force(aspect):
    """Pairs drawn close to contact (thin and thick platelets): the decision
    equals the brute-force one wherever the bounds leave no doubt."""
    rng = np.random.default_rng(int(aspect))
    t = 1.0 / (2 * aspect - 1)  # a = 1, D / (2 t) = aspect
    a = 1.0
    decided = 0
    for _ in range(80):
        ni, nj = rand_units(rng, 2)
        dj = rng.normal(size=3)
        dj *= rng.uniform(0.02, 2.0) / np.linalg.norm(dj)
        lo, up = brute_distance(np.zeros(3), ni, dj, nj, a)
        got = oracle.plt_collide(dj, ni, nj, a, t)
        if up <= 2 * t:
            assert got == 1
            decided += 1
        elif lo > 2 * t:
            assert got == 0
            decided += 1
    assert decided >= 50


def test_coplanar_disks():
    n = np.array([0.0, 0.0, 1.0])
    a, t = 1.0, 0.01
    for ang in np.linspace(0, 2 * math.pi, 7):
        e = np.array([math.cos(ang), math.sin(ang), 0.0])
        assert oracle.plt_collide(e * (2 * a + 2 * t - 1e-9), n, n, a, t) == 1
        assert oracle.plt_collide(e * (2 * a + 2 * t + CLEAR * a), n, n, a, t) == 0
        assert oracle.plt_collide(e * 0.5, n, n, a, t) == 1  # overlapping in the plane


def test_stacked_parallel_disks():
    a, t = 1.0, 0.01
    rng = np.random.default_rng(5)
    for n in rand_units(rng, 10):
        e1, e2 = disk_basis(n)
        for off in (0.0, 0.7, 1.9):
            base = off * e1
            assert oracle.plt_collide(base + n * (2 * t - 1e-12), n, n, a, t) == 1
            assert oracle.plt_collide(base + n * (2 * t + CLEAR * a), n, n, a, t) == 0
            assert oracle.plt_collide(base - n * (2 * t + CLEAR * a), -n, n, a, t) == 0
            # no widening: a gap of 2^-17 a beyond 2 t is a separation
            assert oracle.plt_collide(base + n * (2 * t + 2.0 ** -17 * a), n, n, a, t) == 0


def test_disk_standing_on_disk():
    """Disk j in a vertical plane, lowest point above the interior of disk i
    (horizontal): distance z0 - a."""
    a, t = 1.0, 0.01
    ni = np.array([0.0, 0.0, 1.0])
    for x0, y0 in ((0.0, 0.0), (0.5, -0.3), (-0.2, 0.9)):
        for nj in (np.array([0.0, 1.0, 0.0]), unit([1.0, 1.0, 0.0])):
            z = a + 2 * t
            assert oracle.plt_collide([x0, y0, z - 1e-9], ni, nj, a, t) == 1
            assert oracle.plt_collide([x0, y0, z + CLEAR * a], ni, nj, a, t) == 0


def test_edge_to_edge_right_angle():
    """Disk i horizontal at the origin, disk j in the plane x = x0 centred on
    the x axis: closest points (a, 0, 0) and (x0, 0, 0), distance x0 - a."""
    a, t = 1.0, 0.02
    ni, nj = np.array([0.0, 0.0, 1.0]), np.array([1.0, 0.0, 0.0])
    x0 = a + 2 * t
    assert oracle.plt_collide([x0 - 1e-9, 0, 0], ni, nj, a, t) == 1
    assert oracle.plt_collide([x0 + CLEAR * a, 0, 0], ni, nj, a, t) == 0


def random_rotation(rng):
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q *= np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def test_swap_and_rotation_invariance():
    rng = np.random.default_rng(6)
    a, t = 1.0, 0.05
    n_far = 0
    for _ in range(300):
        ni, nj = rand_units(rng, 2)
        dj = rng.normal(size=3)
        dj *= rng.uniform(0.05, 2.2) / np.linalg.norm(dj)
        c = oracle.plt_collide(dj, ni, nj, a, t)
        assert oracle.plt_collide(-dj, nj, ni, a, t) == c  # exact: the same operations in the midpoint frame
        # rigid rotation: the same answer unless the pair is within 1e-6 of contact
        if oracle.plt_collide(dj, ni, nj, a, t + 1e-6) == oracle.plt_collide(dj, ni, nj, a, t - 1e-6):
            R = random_rotation(rng)
            assert oracle.plt_collide(R @ dj, R @ ni, R @ nj, a, t) == c
            assert oracle.plt_collide(dj, -ni, nj, a, t) == c
            n_far += 1
    assert n_far > 250


def test_unresolved_contact_counts_as_collision():
    """Exactly parallel disks at the threshold: every rim point sits at the
    threshold distance; the decision says collision (closed inequality)."""
    n = np.array([0.0, 0.0, 1.0])
    a, t = 1.0, 0.015625  # 2 t = 1/32, exact
    assert oracle.plt_collide([0.25, 0.0, 2 * t], n, n, a, t) == 1


# --------------------------------------------------------------------------
# System level
# --------------------------------------------------------------------------
def start_config(n, L, a0, t0, seed):
    """Platelets whose bounding spheres do not overlap (so the platelets do
    not either), uniform random normals."""
    rng = np.random.default_rng(seed)
    R = a0 + t0
    X = []
    while len(X) < n:
        p = rng.uniform(0, L, 3)
        ok = True
        for q in X:
            d = p - q
            d -= np.round(d / L) * L
            if d @ d <= (2 * R) ** 2:
                ok = False
                break
        if ok:
            X.append(p)
    return np.array(X), rand_units(rng, n)


def minimage(d, L):
    d = d.copy()
    for k in range(3):
        if d[k] > 0.5 * L[k]:
            d[k] -= L[k]
        if d[k] < -0.5 * L[k]:
            d[k] += L[k]
    return d


def brute_sweep(X, U, box, a0, t0, lam, c_m, c_r, N_l, seed, sweep, collide=None):
    """Alg 3 in the canonical order, each trial tested against every other
    platelet (no cell list), with the reference's contact decision unless
    another predicate is given."""
    collide = collide or oracle.plt_collide
    X, U = X.copy(), U.copy()
    box = np.asarray(box, dtype=np.float64)
    cs = 2.5 * (lam * (a0 + t0)) + c_m
    nc = [3 * max(1, int(box[k] / (3.0 * cs))) for k in range(3)]
    w = [box[k] / nc[k] for k in range(3)]
    cell = [tuple(int(X[i, k] / w[k]) % nc[k] for k in range(3)) for i in range(len(X))]
    a, t = lam * a0, lam * t0
    order = []
    for chi in range(27):
        c0, c1, c2 = chi % 3, (chi // 3) % 3, chi // 9
        for cz in range(c2, nc[2], 3):
            for cy in range(c1, nc[1], 3):
                for cx in range(c0, nc[0], 3):
                    order += [i for i in range(len(X)) if cell[i] == (cx, cy, cz)]
    acc = 0
    for pid in order:
        for l in range(N_l):
            q, u = oracle.plt_trial(seed, sweep, pid, l, box, c_m, c_r, X[pid], U[pid])
            if not any(collide(minimage(X[j] - q, box), u, U[j], a, t)
                       for j in range(len(X)) if j != pid):
                X[pid], U[pid] = q, u
                acc += 1
                break
    return X, U, acc


def test_single_platelet_moves_and_turns():
    box = (1.0, 1.0, 1.0)
    x0 = np.array([[0.5, 0.02, 0.97]])
    u0 = np.array([unit([0.3, -0.4, 0.8])])
    s = oracle.PlateletSystem(box, x0, u0, 0.05, 0.005, c_m=0.05, c_r=0.2, seed=9, sweep=4)
    assert s.sweep() == 1
    X, U = s.state()
    d, _ = oracle.unit_dir_stream(9, 4, 0, 0, 3, 0)
    v, _ = oracle.unit_dir_stream(9, 4, 0, 0, 3, 1)
    expect = [oracle.wrap(x0[0, k] + 0.05 * d[k], 1.0) for k in range(3)]
    np.testing.assert_array_equal(X[0], expect)
    m = u0[0] + 0.2 * v
    np.testing.assert_allclose(U[0], m / np.linalg.norm(m), rtol=0, atol=2e-16)
    assert abs(np.linalg.norm(U[0]) - 1.0) < 4e-16


def test_rotation_streams_independent():
    a = [oracle.unit_dir_stream(5, 7, p, l, 3, 0)[0] for p in range(50) for l in range(3)]
    b = [oracle.unit_dir_stream(5, 7, p, l, 3, 1)[0] for p in range(50) for l in range(3)]
    assert not any(np.array_equal(x, y) for x, y in zip(a, b))
    # stream 0 is the draw of the spheres
    np.testing.assert_array_equal(a[4], oracle.unit_dir(5, 7, 1, 1, 3)[0])


@pytest.mark.parametrize("c_r", [0.0, 0.3])
def test_sweep_equals_brute_force_sweep(c_r):
    box = (1.0, 1.2, 1.0)
    a0, t0 = 0.09, 0.01
    X0, U0 = start_config(40, np.array(box), a0, t0, 11)
    lam, c_m = 1.4, 0.04
    s = oracle.PlateletSystem(box, X0, U0, a0, t0, lam=lam, c_m=c_m, c_r=c_r, N_l=4, seed=21, sweep=2)
    X, U = X0, U0
    for k in range(2):
        X, U, acc = brute_sweep(X, U, box, a0, t0, lam, c_m, c_r, 4, 21, 2 + k)
        assert s.sweep() == acc
        SX, SU = s.state()
        np.testing.assert_array_equal(SX, X)
        np.testing.assert_array_equal(SU, U)
    assert s.sweep_counter == 4


def test_check_against_brute_force_pairs():
    rng = np.random.default_rng(12)
    box = np.array([1.0, 1.0, 1.0])
    a0, t0 = 0.08, 0.01
    X = rng.uniform(0, 1, (120, 3))
    U = rand_units(rng, 120)
    s = oracle.PlateletSystem(box, X, U, a0, t0)
    cnt, flags = s.check()
    ij, npairs = oracle.plt_pairs_brute(box, X, U, a0, t0)
    ref = np.zeros(120, dtype=np.uint8)
    ref[ij.reshape(-1)] = 1
    assert npairs > 5
    np.testing.assert_array_equal(flags, ref)
    assert cnt == int(ref.sum())
    # independent check of the pairs: each brute-force pair is within the
    # brute-force distance bound, pairs far apart are absent
    for i, j in ij[:10]:
        _, up = brute_distance(X[i], U[i], X[i] + minimage(X[j] - X[i], box), U[j], a0)
        assert up <= 2 * t0 + 1e-3


def test_iterations_keep_p_collision_free_and_reach_density():
    box = np.array([1.0, 1.0, 1.0])
    a0, t0 = 0.02, 0.002
    n = 150
    X0, U0 = start_config(n, box, a0 * 2.2, t0 * 2.2, 13)
    rho_t = 1.0
    lam_t = oracle.plt_lambda_for_density(box, n, a0, t0, rho_t)
    D = 2 * lam_t * (a0 + t0)
    assert n * D ** 3 / 1.0 == pytest.approx(rho_t, rel=1e-14)  # Eq. 1
    s = oracle.PlateletSystem(box, X0, U0, a0, t0, lam=1.0, lam_t=lam_t, c_w=0.15, c_m=0.01, c_r=0.1, N_l=6,
                              seed=5)
    m = 0
    for _ in range(40):
        acc, info = s.iterate()
        if acc == 2:
            break
        m += acc
        _, npairs = s.pairs_brute()
        assert npairs == 0
        if s.lam < lam_t:
            assert s.lam == pytest.approx(1.15 ** m, rel=1e-13)
    assert s.lam == lam_t


def test_rejected_swell_is_discarded_and_p_shaken():
    """Two coaxial platelets whose gap one swell step closes, with steps far
    too short to reopen it: every round of the N_k loop leaves them in
    contact, the swollen state is discarded, P (at the old scale) is swept
    N_shake times, the scale stays and P stays collision-free (Alg 1)."""
    a0, t0 = 0.1, 0.01
    n = np.array([0.0, 0.0, 1.0])
    x = np.array([[1.0, 1.0, 1.0], [1.0, 1.0, 1.0 + 2 * t0 * 1.005]])
    u = np.stack([n, n])
    s = oracle.PlateletSystem((2.0, 2.0, 2.0), x, u, a0, t0, lam=1.0, lam_t=2.0, c_w=0.01, c_m=1e-7, c_r=0.0,
                              N_k=4, N_l=3, N_shake=5, seed=3)
    acc, info = s.iterate()
    assert acc == 0
    assert info == dict(k_sweeps=4, overlapping=2, shake_sweeps=5)
    assert s.lam == 1.0 and s.sweep_counter == 4 + 5
    assert s.counters()["shaken"] == 1
    _, npairs = s.pairs_brute()
    assert npairs == 0
    X, U = s.state()
    np.testing.assert_array_equal(U, u)  # no rotation with c_r = 0
    assert np.all(np.abs(X - x) <= 5 * 1e-7 + 1e-15)  # each sweep moves a platelet at most c_m


def neighbour_alignment(X, U, D):
    """Mean |n_i . n_j| over the pairs of centres closer than D (periodic
    unit box); 1/2 for independent uniform orientations."""
    tree = spatial.cKDTree(X, boxsize=1.0)
    p = tree.query_pairs(D, output_type="ndarray")
    return float(np.mean(np.abs(np.sum(U[p[:, 0]] * U[p[:, 1]], axis=1))))


def test_relaxation_aligns_neighbours():
    """Section 3.3 (Fig. 8): fast swelling with short steps gives a "house of
    cards" whose neighbours are oriented at random; relaxing it with zero
    swelling and longer steps and turns grows domains of nearly parallel
    platelets.  600 platelets of aspect ratio 100 to number density 5, then
    150 relaxation sweeps; both states collision-free."""
    import srm_inputs
    w = srm_inputs.platelets(n=600, seed=7, rho_t=5.0)
    D = w.extra["D"]
    s = oracle.PlateletSystem(w.box, w.x, w.u, w.a0, w.t0, lam=w.lambda0, lam_t=1.0, c_w=w.c_w, c_m=w.c_m,
                              c_r=w.c_r, seed=w.seed)
    s.run()
    assert s.lam == 1.0 and s.pairs_brute()[1] == 0
    X, U = s.state()
    hoc = neighbour_alignment(X, U, D)
    r = oracle.PlateletSystem(w.box, X, U, w.a0, w.t0, lam=1.0, lam_t=1.0, c_w=0.0, c_m=0.1 * D, c_r=0.1,
                              seed=w.seed, sweep=s.sweep_counter)
    for _ in range(150):
        r.sweep()
    assert r.pairs_brute()[1] == 0
    X, U = r.state()
    relaxed = neighbour_alignment(X, U, D)
    assert abs(hoc - 0.5) < 0.03, hoc
    assert relaxed > hoc + 0.06, (hoc, relaxed)


def test_decision_monotone_in_threshold():
    """A larger half-thickness never turns a contact into a separation: the
    bisection prunes fewer intervals and keeps every hit (the flip-threshold
    bisection of the pins above relies on this)."""
    rng = np.random.default_rng(31)
    ts = np.geomspace(1e-4, 0.3, 25)
    for _ in range(150):
        ni, nj = rand_units(rng, 2)
        dj = rng.normal(size=3)
        dj *= rng.uniform(0.0, 2.4) / np.linalg.norm(dj)
        got = [oracle.plt_collide(dj, ni, nj, 1.0, t) for t in ts]
        assert all(a <= b for a, b in zip(got, got[1:])), got


def test_rim_search_resolves_near_contacts_within_budget():
    """The rim search decides near-contacts (thresholds 1e-4 and 1e-6 of
    the rim's distance to the other disk away from it; thin and thick,
    near-parallel and crossing disks) by its bound, well below its safety cap
    of 2^20 evaluations per rim.  (A first-order bound needs about
    1/sqrt(gap) arcs near a flat minimum, so the count grows as the gap
    shrinks; the cap bounds it.)"""
    rng = np.random.default_rng(41)
    worst = {1e-4: 0, 1e-6: 0}
    for _ in range(60):
        ni, nj = rand_units(rng, 2)
        if rng.uniform() < 0.3:
            nj = unit(ni + 1e-3 * rng.normal(size=3))
        dj = rng.normal(size=3)
        dj *= rng.uniform(0.05, 2.1) / np.linalg.norm(dj)
        # the rim's distance to the other disk, by bisection on the threshold
        hi, lo = 4.0, 0.0
        for _ in range(45):
            mid = 0.5 * (hi + lo)
            if oracle.plt_rim_near_disk(-0.5 * dj, ni, 1.0, 0.5 * dj, nj, 1.0, mid)[0]:
                hi = mid
            else:
                lo = mid
        for eps in worst:
            # (lo = 0: the disks cross, every threshold is a contact)
            for thr, expect in ((hi * (1 + eps), 1), (lo * (1 - eps), 0))[:2 if lo > 0 else 1]:
                got, ev = oracle.plt_rim_near_disk(-0.5 * dj, ni, 1.0, 0.5 * dj, nj, 1.0, thr)
                assert got == expect
                worst[eps] = max(worst[eps], ev)
    assert worst[1e-4] < 1 << 13 and worst[1e-6] < 1 << 16, worst
