"""Platelets (spherodisks, Section 3.3) on the GPU through the C interface
(include/srm_platelet.h).

The kernel decides contact in binary32 against 2 t + 2^-16 a (the kernel
specification, tests/plt_kernel_spec.c), the reference in binary64 against
2 t.  Two comparisons follow:
  * bit for bit with the reference run on the kernel specification's
    predicate: the contact decision on many pairs, sweeps with and without
    rotation, whole iterations of Algorithm 1 (accepted and rejected),
    Algorithm 6 on a configuration full of collisions, a run to target, the
    edge cases (one platelet, three cells per axis);
  * one-sided with the binary64 reference itself: every contact of the
    reference is a contact of the kernel, every contact only the kernel
    reports is within the widening of touching (or, where a bisection ran
    out of budget, within 2^-12 a); after a sweep every pair the
    reference finds colliding consists of platelets that did not move; final
    states have no colliding pair by the reference's brute force.
Plus the bounded wait and a full-size run."""

import numpy as np
import pytest

import oracle
import plt_kernel_spec as spec
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def rand_units(rng, n):
    v = rng.normal(size=(n, 3))
    return v / np.linalg.norm(v, axis=1, keepdims=True)


def pair_set(seed, m, a, t):
    rng = np.random.default_rng(seed)
    ni, nj = rand_units(rng, m), rand_units(rng, m)
    d = rand_units(rng, m) * rng.uniform(0.0, 2 * a + 3 * t, (m, 1))
    # a quarter nearly parallel (stacks), an eighth exactly parallel
    k = m // 4
    nj[:k] = ni[:k] + 0.01 * rng.normal(size=(k, 3))
    nj[:k] /= np.linalg.norm(nj[:k], axis=1, keepdims=True)
    nj[k:k + k // 2] = ni[k:k + k // 2]
    return d, ni, nj


@pytest.mark.parametrize("a,t", [(1.0, 1.0 / 199.0), (1.0, 0.1), (0.03, 0.0003)])
def test_pair_decisions(a, t):
    """60 000 decisions in all (three sizes): equal to the kernel
    specification bit for bit; one-sided against the binary64 reference."""
    m = 20000
    d, ni, nj = pair_set(int(1 / t), m, a, t)
    got = srm.srm_plt_collide_pairs(d, ni, nj, a, t)
    want = np.array([spec.collide32(d[k], ni[k], nj[k], a, t) for k in range(m)], dtype=np.uint8)
    np.testing.assert_array_equal(got, want)
    ref = np.array([oracle.plt_collide(d[k], ni[k], nj[k], a, t) for k in range(m)], dtype=np.uint8)
    assert 0.05 < ref.mean() < 0.95
    assert np.all(got[ref == 1] == 1), "a binary64 contact the kernel misses"
    extra = np.nonzero((got == 1) & (ref == 0))[0]
    assert all(spec.confirmed_by_reference(oracle, d[k], ni[k], nj[k], a, t) for k in extra)


def small_workload(n, seed, aspect=20.0, rho_t=3.0, **kw):
    return srm_inputs.platelets(seed=seed, n=n, aspect=aspect, rho_t=rho_t, **kw)


def both(w, lam0=None, lam_t=1.0, gpu_kw=None, **kw):
    """The GPU handle and the reference on the kernel specification's
    contact predicate, on the same start."""
    lam0 = w.lambda0 if lam0 is None else lam0
    args = dict(c_w=w.c_w, c_m=w.c_m, c_r=w.c_r)
    args.update(kw)
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, lam0, lam_t, w.seed, **args, **(gpu_kw or {}))
    o = oracle.PlateletSystem(w.box, w.x, w.u, w.a0, w.t0, lam=lam0, lam_t=lam_t, seed=w.seed,
                              contact=spec.address(), **args)
    return g, o


def binary64_pairs(box, x, u, a, t):
    """Colliding pairs by the binary64 reference's brute force, as a set."""
    ij, n = oracle.plt_pairs_brute(box, x, u, a, t, cap=1 << 20)
    assert n == len(ij)
    return {(int(i), int(j)) for i, j in ij}


def assert_sweep_one_sided(box, x0, u0, x1, u1, a, t):
    """After a sweep: every pair the binary64 reference finds colliding is
    a pair of platelets that did not move (a moved platelet's new place was
    free by the kernel's wider test, hence by the reference's), and it
    collided before the sweep too."""
    moved = np.any(x1 != x0, axis=1) | np.any(u1 != u0, axis=1)
    after = binary64_pairs(box, x1, u1, a, t)
    assert not any(moved[i] or moved[j] for i, j in after)
    assert after <= binary64_pairs(box, x0, u0, a, t)
    return int(moved.sum())


def assert_same_state(g, o):
    gx, gu, info = g.state()
    ox, ou = o.state()
    np.testing.assert_array_equal(gx, ox)
    np.testing.assert_array_equal(gu, ou)
    assert info["lambda_"] == o.lam
    assert info["sweep"] == o.sweep_counter


@pytest.mark.parametrize("c_r,kernel", [(0.0, 0), (0.05, 0), (0.05, 1)])
def test_sweeps_bit_exact(c_r, kernel):
    """Kernel 0: a block per cell with the 27 cells around it in shared
    memory (this grid qualifies); kernel 1: a warp per cell."""
    w = small_workload(3000, 11)
    # sweeps at 2.5 times the starting size, where neighbours interact
    lam = 2.5 * w.lambda0
    g, o = both(w, lam0=lam, c_m=0.05 * w.extra["D"], c_r=c_r, gpu_kw=dict(sweep_kernel=kernel))
    a, t = lam * w.a0, lam * w.t0
    for _ in range(3):
        x0, u0, _ = g.state()
        assert g.sweeps(1) == o.sweep()
        assert_same_state(g, o)
        x1, u1, _ = g.state()
        assert assert_sweep_one_sided(w.box, x0, u0, x1, u1, a, t) > 50
    st = g.sweep_stats()
    assert (st["staged_sweeps"], st["warp_sweeps"]) == ((3, 0) if kernel == 0 else (0, 3))
    assert st["unstaged_cells"] == 0
    g.close()


def test_staged_sweep_overflow_matches_warp_kernel():
    """A cluster of 1500 overlapping platelets inside a few cells: the 27
    cells around those cells hold more than the 1024 platelets the block
    kernel stages, so it moves them from global memory; both kernels end
    bit for bit alike, and equal the reference on one sweep."""
    rng = np.random.default_rng(21)
    n_bg, n_cl = 1500, 1500
    # cells of width 1/18: the 27 cells around the cluster's centre hold it all
    x = np.concatenate([rng.uniform(0, 1, (n_bg, 3)), 0.5 + rng.uniform(-0.05, 0.05, (n_cl, 3))])
    u = rand_units(rng, n_bg + n_cl)
    a0, t0, c_m = 0.02, 0.0005, 0.004
    runs = []
    for kernel in (0, 1):
        g = srm.Platelets((1, 1, 1), x, u, a0, t0, 1.0, 1.0, 5, c_m=c_m, c_r=0.05, sweep_kernel=kernel)
        moved = g.sweeps(2)
        xs, us, _ = g.state()
        runs.append((xs, us, moved, g.sweep_stats()))
        g.close()
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    np.testing.assert_array_equal(runs[0][1], runs[1][1])
    assert runs[0][2] == runs[1][2] > 0
    assert runs[0][3]["staged_sweeps"] == 2 and runs[0][3]["unstaged_cells"] > 0
    assert runs[1][3]["warp_sweeps"] == 2
    g = srm.Platelets((1, 1, 1), x, u, a0, t0, 1.0, 1.0, 5, c_m=c_m, c_r=0.05)
    o = oracle.PlateletSystem((1, 1, 1), x, u, a0, t0, c_m=c_m, c_r=0.05, seed=5, contact=spec.address())
    assert g.sweeps(1) == o.sweep()
    assert_same_state(g, o)
    g.close()


def test_iterations_bit_exact_with_rejections():
    """Fast swelling against short steps: some iterations are discarded and
    P is shaken; every iteration's outcome and state match."""
    w = small_workload(1500, 12, aspect=50.0, rho_t=4.0, c_w=0.04, c_m_rel=0.02, c_r=0.01)
    g, o = both(w, N_k=3, N_shake=2)
    results = []
    for _ in range(25):
        gi = g.step()
        acc, oi = o.iterate()
        results.append(acc)
        assert gi["result"] == acc
        if acc != 2:
            assert gi["k_sweeps"] == oi["k_sweeps"]
            assert gi["colliding"] == oi["overlapping"]
            assert gi["shake_sweeps"] == oi["shake_sweeps"]
        assert_same_state(g, o)
    assert 0 in results and 1 in results
    x, u, st = g.state()
    assert not binary64_pairs(w.box, x, u, st["lambda_"] * w.a0, st["lambda_"] * w.t0)
    g.close()


def test_run_to_target_bit_exact():
    w = small_workload(800, 13, aspect=100.0, rho_t=2.0)
    g, o = both(w)
    info = g.run_to_target()
    o.run()
    assert info["converged"] == 1
    assert_same_state(g, o)
    assert info["rho"] == pytest.approx(2.0, rel=1e-12)
    assert g.check()[0] == 0
    _, npairs = o.pairs_brute()
    assert npairs == 0
    g.close()


@pytest.mark.parametrize("kernel", [0, 1])
def test_check_flags_bit_exact(kernel):
    """Kernel 0: a block per cell with the staged neighbourhood (this grid
    qualifies); kernel 1: a thread per platelet."""
    rng = np.random.default_rng(14)
    n = 4000
    x = rng.uniform(0, 1, (n, 3))
    u = rand_units(rng, n)
    a0, t0 = 0.02, 0.002
    g = srm.Platelets((1, 1, 1), x, u, a0, t0, 1.0, 1.0, 3, c_m=0.001, sweep_kernel=kernel)
    cnt, flags = g.check()
    o = oracle.PlateletSystem((1, 1, 1), x, u, a0, t0, contact=spec.address())
    ocnt, oflags = o.check()
    np.testing.assert_array_equal(flags, oflags)
    assert cnt == ocnt and 0.05 * n < cnt < 0.95 * n
    # one-sided: every platelet the binary64 reference flags is flagged
    rcnt, rflags = oracle.PlateletSystem((1, 1, 1), x, u, a0, t0).check()
    assert np.all(flags[rflags == 1] == 1) and rcnt <= cnt
    g.close()


@pytest.mark.parametrize("kernel", [0, 1])
def test_three_cells_per_axis_and_single_platelet(kernel):
    w = small_workload(60, 15, aspect=10.0, rho_t=1.0)
    c_m = 0.05 * w.extra["D"]
    g, o = both(w, lam0=1.0, c_m=c_m, c_r=0.1, gpu_kw=dict(sweep_kernel=kernel))
    assert list(oracle.grid(3, w.box, 1.0, w.a0 + w.t0, c_m)[0]) == [3, 3, 3]
    for _ in range(2):
        assert g.sweeps(1) == o.sweep()
    assert_same_state(g, o)
    if kernel == 0:
        assert g.sweep_stats()["staged_sweeps"] == 2
    g.close()
    x = np.array([[0.5, 0.999, 0.001]])
    u = np.array([[0.0, 0.6, 0.8]])
    g = srm.Platelets((1, 1, 1), x, u, 0.05, 0.005, 1.0, 1.0, 4, c_m=0.01, c_r=0.3)
    o = oracle.PlateletSystem((1, 1, 1), x, u, 0.05, 0.005, c_m=0.01, c_r=0.3, seed=4)
    assert g.sweeps(1) == 1 == o.sweep()
    assert_same_state(g, o)
    g.close()


def test_bounded_wait_reports_timeout():
    w = small_workload(2000, 16)
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, w.lambda0, 1.0, w.seed, c_m=w.c_m, wait_limit=-1)
    with pytest.raises(srm.SrmError) as e:
        g.sweeps(1)
    assert e.value.status == 5
    g.close()
    h = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, w.lambda0, 1.0, w.seed, c_m=w.c_m)
    assert h.sweeps(2) > 0
    h.close()


def test_full_size_house_of_cards_then_relaxation():
    """20000 platelets of aspect ratio 100 to number density 5 (the paper's
    largest case), then relaxation sweeps with zero swelling and a larger
    step: collision-free by the reference's brute force over every pair, at
    the number density of Eq. 1."""
    w = srm_inputs.platelets()
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, w.lambda0, 1.0, w.seed, c_w=w.c_w, c_m=w.c_m, c_r=w.c_r)
    info = g.run_to_target(4000)
    assert info["converged"] == 1
    assert info["rho"] == pytest.approx(5.0, rel=1e-12)
    g.set_params(c_w=0.0, c_m=0.1 * w.extra["D"], c_r=0.1)
    assert g.sweeps(20) > 0
    x, u, st = g.state()
    assert g.check()[0] == 0
    _, npairs = oracle.plt_pairs_brute(w.box, x, u, st["lambda_"] * w.a0, st["lambda_"] * w.t0)
    assert npairs == 0
    np.testing.assert_allclose(np.linalg.norm(u, axis=1), 1.0, atol=1e-14)
    g.close()
