"""Parity of the CUDA path (through the C interface) with the FP64 reference.

FP64 form: every iteration, sweep and pair list must equal the reference bit
for bit on the same inputs -- the path evaluates the same IEEE operations in
an order that provably gives the same result (coloured sweep, exact
collision predicate).  FP32 form: tolerance 1e-5 of the mean radius for one
sweep, and overlap-free FP64 certification of full runs.
"""
import math

import numpy as np
import pytest

import oracle
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def pair(w, precision=64, literal=False, **kw):
    args = dict(c_w=w.c_w, c_m=w.c_m, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake)
    args.update(kw)
    lam0 = args.pop("lambda0", 1.0)
    lam_t = args.pop("lambda_t", None)
    gpu_only = {k: args.pop(k) for k in ("wait_limit",) if k in args}
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                precision=precision, lambda0=lam0, lambda_t=lam_t or 0.0, **args, **gpu_only)
    o = oracle.System(w.dim, w.box, w.x, w.radii, lam=lam0, lam_t=lam_t,
                      target_phi=None if lam_t else w.target_phi, seed=w.seed, literal=literal,
                      **args)
    return g, o


def assert_same_state(g, o):
    x, R = g.positions()
    np.testing.assert_array_equal(x, o.x)
    st = g.state()
    assert st["lambda"] == o.lam
    np.testing.assert_array_equal(R, o.radii())
    assert st["sweep"] == o.sweep_counter


def small_3d(n=2000, phi_t=0.45, seed=7):
    return srm_inputs._mono("spheres_small", 3, n, phi_t, 0.1, seed)


@pytest.mark.parametrize("maker", [lambda: srm_inputs.disks_1k(), lambda: small_3d()])
def test_fp64_iterations_bit_exact(maker):
    w = maker()
    g, o = pair(w)
    assert g.state()["lambda_t"] == o.lambda_for_phi(w.target_phi)
    for _ in range(12):
        gi = g.step()
        acc, oi = o.iterate()
        assert gi["result"] == acc
        assert gi["k_sweeps"] == oi["k_sweeps"]
        if acc == 0:
            assert gi["overlapping"] == oi["overlapping"]
        assert_same_state(g, o)


@pytest.mark.parametrize("maker", [lambda: srm_inputs.disks_1k(), lambda: small_3d(1500, 0.40)])
def test_fp64_full_run_bit_exact(maker):
    w = maker()
    g, o = pair(w)
    info = g.run_to_target()
    o.run()
    assert info["converged"]
    assert_same_state(g, o)
    c = o.counters()
    assert info["iterations"] == c["iters"] and info["sweeps"] == c["sweeps"]
    assert info["accepted"] == c["accepted"] and info["shaken"] == c["shaken"]
    pairs, gap, phi = g.certify()
    assert pairs == 0 and gap > 0
    assert abs(phi - w.target_phi) < 1e-9
    assert oracle.pairs_brute(w.dim, w.box, *g.positions())[1] == 0


@pytest.mark.parametrize("dim", [2, 3])
def test_pair_sets_and_sweeps_bit_exact(dim):
    """Swell a clean state so that it overlaps, then compare the colliding
    pair set (Algorithm 6 over pairs) and single sweeps of Algorithm 3."""
    w = srm_inputs._mono("swollen", dim, 1200 if dim == 2 else 1500, 0.4, 0.2, 11 + dim)
    g, o = pair(w, c_m=0.2 * w.radii[0])
    for lam in (1.12, 1.25):
        g.set_scale(lam)
        o.lam = lam
        for _ in range(3):
            gp, op = g.overlap_pairs(), o.pairs()
            assert len(op) > 0
            np.testing.assert_array_equal(gp, op)
            np.testing.assert_array_equal(gp, oracle.pairs_brute(dim, w.box, o.x, o.radii())[0])
            moved = g.sweep(1)
            assert moved == o.sweep()
            assert_same_state(g, o)


def test_edge_single_particle():
    box = (1.0, 0.7, 1.3)
    x = np.array([[0.999, 0.01, 0.5]])
    w = srm_inputs.Workload("one", 3, box, np.array([0.05]), x, 0.001, 99, c_m=0.03)
    g, o = pair(w, c_w=0.05)
    for _ in range(5):
        g.step()
        o.iterate()
        assert_same_state(g, o)
    assert g.overlap_pairs().shape == (0, 2)


def test_edge_three_cells_rectangular_polydisperse():
    """Few large particles: 3 cells on some axis, unequal box sides, radii
    spread over 2x, a ragged particle count."""
    rng = np.random.default_rng(5)
    n = 37
    box = (1.0, 0.8, 1.6)
    r = rng.uniform(0.05, 0.1, size=n) * 0.6
    x = srm_inputs.rsa(3, box, r, 5)
    w = srm_inputs.Workload("few", 3, box, r, x, 0.05, 5, c_m=0.01)
    g, o = pair(w, c_w=0.02)
    for _ in range(20):
        g.step()
        o.iterate()
        assert_same_state(g, o)


def test_edge_shake_path():
    """A swelling rate too large for N_k sweeps: discard and shake."""
    w = srm_inputs._mono("shake", 2, 900, 0.6, 0.45, 21)
    g, o = pair(w, c_w=0.2, N_k=2, N_l=3, N_shake=3)
    for _ in range(4):
        gi = g.step()
        acc, oi = o.iterate()
        assert gi["result"] == acc
        assert gi["k_sweeps"] == oi["k_sweeps"]
        assert gi["overlapping"] == oi["overlapping"]
        assert_same_state(g, o)
    assert o.counters()["shaken"] > 0


def test_edge_jammed_lattice():
    m = 12
    a = 1.0 / m
    gx = (np.arange(m) + 0.5) * a
    X = np.array([(x, y) for y in gx for x in gx])
    R = np.full(m * m, 0.5 * a * (1 - 1e-9))
    w = srm_inputs.Workload("lattice", 2, (1.0, 1.0), R, X, 0.9, 3, c_m=0.05 * a)
    g, o = pair(w)
    assert g.sweep(1) == 0 == o.sweep()
    assert_same_state(g, o)


MARGIN = 1e-5  # relative decision margin within which the FP32 guard band may decide otherwise


def fp32_sweep_check(w, lam, c_m, sweeps=1, tuning=None):
    """Sweeps in the FP32 cell-relative form against the FP64 reference on the
    same state and draws, every particle's position compared with tolerance
    1e-5 of the mean radius.

    The FP32 form may decide a trial differently only where the reference's
    decision lay within MARGIN (relative) of contact: its guard band (4e-6 on
    the squared distance) and the binary32 rounding of its offsets amount to
    about 3e-6.  A changed decision moves that particle elsewhere, and the
    sweep carries the change to neighbours handled later, within one
    interaction range (2 R_max + 2 c_m, plus the moves) per link.  So every
    particle out of tolerance must belong to a connected group -- particles
    out of tolerance or with a near-contact decision, linked when their
    starting positions are within that range -- that holds a near-contact
    decision, and there must be no more of them than such decisions allow
    (MAX_PER_ROOT per root).  Returns (fraction within tolerance, out of
    tolerance, roots)."""
    spatial = pytest.importorskip("scipy.spatial")
    g, o = pair(w, precision=32, c_m=c_m)
    if tuning:
        g.set_tuning(*tuning)
    g.set_scale(lam)
    o.lam = lam
    o.track_margins(True)
    box = np.array(w.box, dtype=float)
    x0 = o.x.copy()
    roots = np.zeros(w.n, dtype=bool)
    for _ in range(sweeps):
        g.sweep(1)
        o.sweep()
        roots |= o.margins < MARGIN
    xg, _ = g.positions()
    xo = o.x
    d = xg - xo
    d = d - np.round(d / box) * box
    rbar = float(np.mean(o.radii()))
    err = np.sqrt(np.sum(d * d, axis=1))
    bad = err >= 1e-5 * rbar
    nb, nr = int(bad.sum()), int(roots.sum())
    if nb:
        assert nr > 0, "divergence without a near-contact decision"
        nodes = np.nonzero(bad | roots)[0]
        link = 2 * float(np.max(o.radii())) + 2 * c_m * (1 + sweeps)
        pairs = spatial.cKDTree(np.mod(x0[nodes], box), boxsize=box).query_pairs(link, output_type="ndarray")
        parent = np.arange(len(nodes))

        def find(i):
            while parent[i] != i:
                parent[i] = parent[parent[i]]
                i = parent[i]
            return i
        for i, j in pairs:
            ri, rj = find(i), find(j)
            if ri != rj:
                parent[ri] = rj
        comp = np.array([find(i) for i in range(len(nodes))])
        has_root = set(comp[roots[nodes]])
        lonely = [int(nodes[i]) for i in range(len(nodes)) if bad[nodes[i]] and comp[i] not in has_root]
        assert not lonely, f"particles out of tolerance with no near-contact decision in reach: {lonely[:5]}"
        assert nb <= MAX_PER_ROOT * nr, (nb, nr)
    assert nr <= max(10, 0.002 * w.n), nr
    return 1.0 - nb / w.n, nb, nr


MAX_PER_ROOT = 4


@pytest.mark.parametrize("seed,dim", [(13, 3), (14, 3), (15, 2)])
def test_fp32_sweep_within_tolerance(seed, dim):
    w = small_3d(3000, 0.40, seed=seed) if dim == 3 else srm_inputs._mono("d2", 2, 3000, 0.5, 0.1, seed)
    frac, _, _ = fp32_sweep_check(w, 1.15, 0.3 * w.radii[0])
    assert frac > 0.99


@pytest.mark.parametrize("lam,sweeps,tuning", [(1.0, 1, None), (1.08, 2, None), (1.08, 2, (0, 0, 1)),
                                               (1.08, 2, (1, 64))])
def test_fp32_sweep_polydisperse_clustered(lam, sweeps, tuning):
    # log-normal radii and a clustered start: dense cluster cores give cells
    # with many particles and staged candidate lists of several 32-wide chunks;
    # the default kernel there has the staged path, (0, 0, 1) selects the one
    # with the general path only, and a staging capacity of 64 sends the
    # cells to the general path (overflowing its staging)
    w = srm_inputs.poly_1m(n=20000)
    frac, _, _ = fp32_sweep_check(w, lam, w.c_m, sweeps=sweeps, tuning=tuning)
    assert frac > 0.99


@pytest.mark.parametrize("maker", [lambda: srm_inputs.poly_1m(n=20000), lambda: small_3d(3000, 0.45),
                                   lambda: srm_inputs.disks_1k()])
def test_fp32_sweep_kernels_agree_bit_for_bit(maker):
    """The two FP32 sweep kernels (general path only; with the staged path)
    and an overflowing staging capacity evaluate the same binary32
    operations on the same candidates: iterations agree bit for bit."""
    w = maker()
    runs = []
    for tuning in ((0, 0, 1), (0, 0, 2), (1, 64, 2)):
        g, _ = pair(w, precision=32)
        g.set_tuning(*tuning)
        assert g.tuning()["sweep_path"] == tuning[2]
        infos = [g.step() for _ in range(5)]
        runs.append((g.positions()[0], [(i["result"], i["k_sweeps"]) for i in infos], g.state()["sweep"]))
        g.close()
    for x, it, sw in runs[1:]:
        np.testing.assert_array_equal(x, runs[0][0])
        assert it == runs[0][1] and sw == runs[0][2]


def test_fp64_has_no_staged_sweep_kernel():
    g, _ = pair(small_3d(500, 0.3))
    assert g.tuning()["sweep_path"] == 1
    with pytest.raises(srm.SrmError):
        g.set_tuning(0, 0, 2)
    g.close()


@pytest.mark.parametrize("capacity", [0, 64])
def test_fp64_clustered_polydisperse_iterations_bit_exact(capacity):
    """The benchmark's input at 20 000 spheres (log-normal radii, 200
    Gaussian clusters), FP64 form: every iteration equals the reference bit
    for bit -- with the default staging capacity (whole stencils staged),
    and with capacity 64, which sends every cell through the general path
    and overflows its staging."""
    w = srm_inputs.poly_1m(n=20000)
    g, o = pair(w)
    if capacity:
        g.set_tuning(1, capacity)
    for _ in range(6):
        gi = g.step()
        acc, oi = o.iterate()
        assert gi["result"] == acc and gi["k_sweeps"] == oi["k_sweeps"]
        assert_same_state(g, o)
    if capacity:
        assert g.state()["stage_overflow"] > 0


def bimodal_dense(n_big=24, per=120, seed=31, L=36.0):
    """3D: large spheres (R = 2), each ringed by `per` small ones (R = 0.4)
    in a shell of radii 2.41 .. 3.1, in a box of 6 x 6 x 6 cells; c_m = 0.8:
    a large sphere's near list (centres within R + R_t + c_m = 3.2) holds
    `per` > 64 small spheres, and its stencil far exceeds a staging capacity
    of 64."""
    rng = np.random.default_rng(seed)
    big = []
    while len(big) < n_big:
        p = rng.uniform(0, L, 3)
        d = np.array(big) - p if big else np.zeros((0, 3))
        d -= np.round(d / L) * L
        if not big or np.min(np.sum(d * d, axis=1)) >= 9.0 ** 2:
            big.append(p)
    small = []
    for c in big:
        mine = []
        for _ in range(20000):
            if len(mine) >= per:
                break
            v = rng.normal(size=3)
            q = c + v / np.linalg.norm(v) * rng.uniform(2.41, 3.1)
            if not mine or np.min(np.sum((np.array(mine) - q) ** 2, axis=1)) > 0.8 ** 2 * (1 + 1e-9):
                mine.append(q)
        small += mine
    x = np.mod(np.array(big + small), L)
    r = np.concatenate([np.full(n_big, 2.0), np.full(len(small), 0.4)])
    return srm_inputs.Workload("bimodal", 3, (L, L, L), r, x, 0.35, seed, c_m=0.8)


def test_fp64_near_list_overflow_bit_exact():
    """Stencils far beyond the staging capacity (64) and near lists beyond
    theirs: the general path reads the unstaged candidates from global
    memory and tests those particles' trials against every candidate; both
    sweeps equal the reference bit for bit (and the state counters show
    that both fallbacks ran)."""
    w = bimodal_dense()
    assert oracle.grid(3, w.box, 1.02, 2.0, w.c_m)[0].tolist() == [6, 6, 6]
    g, o = pair(w, wait_limit=1 << 26)
    g.set_tuning(1, 64)
    g.set_scale(1.02)
    o.lam = 1.02
    for _ in range(2):
        assert g.sweep(1) == o.sweep()
        assert_same_state(g, o)
    st = g.state()
    assert st["stage_overflow"] > 0 and st["near_fallback"] > 0


@pytest.mark.parametrize("maker", [lambda: srm_inputs.disks_1k(), lambda: small_3d(3000, 0.45)])
def test_fp32_full_run_certifies(maker):
    w = maker()
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                precision=32, c_m=w.c_m, c_w=w.c_w)
    info = g.run_to_target()
    assert info["converged"]
    pairs, gap, phi = g.certify()
    assert pairs == 0 and gap > 0 and abs(phi - w.target_phi) < 1e-9
    x, R = g.positions()
    assert oracle.certify(w.dim, w.box, x, R)[0] == 0


def test_rsa_init_through_c_interface():
    g = srm.Rve(3, (1.0, 1.0, 1.0), ("mono", 1.0), 0.3, 4, n=5000, c_m=0.002, init="rsa", f0=0.1)
    st = g.state()
    assert abs(st["phi"] - 0.1) < 1e-12
    x, R = g.positions()
    assert oracle.certify(3, (1.0, 1.0, 1.0), x, R)[0] == 0
    info = g.run_to_target()
    assert info["converged"] and g.certify()[0] == 0
