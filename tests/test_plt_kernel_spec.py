"""The platelet kernel specification (the CUDA kernel's binary32 contact
decision, tests/plt_kernel_spec.c) against the binary64 reference, on the CPU.

The specification decides contact against 2 t + 2^-16 a in binary32, so it
must find every contact of the reference (distance <= t_i + t_j).  Every
contact only it reports must lie within the widening (plus the binary32
rounding of its inputs) of touching -- the reference reports contact for it
at a threshold raised by 1.25 x 2^-16 a -- or be a near-contact whose
bisection ran out of budget (counted as contact by the kernel), within
2^-12 a of touching.  Plus: the reference's sweep run on the
specification's predicate equals a brute-force sweep on the same predicate,
which is what the GPU sweeps are compared with bit for bit."""
import numpy as np
import pytest

import oracle
import plt_kernel_spec as spec
from test_oracle_platelet import brute_sweep, rand_units, start_config



def pair_set(seed, m, a, t):
    """Random pairs with centre distances up to 2 a + 3 t; a quarter nearly
    parallel (stacks), an eighth exactly parallel."""
    rng = np.random.default_rng(seed)
    ni, nj = rand_units(rng, m), rand_units(rng, m)
    d = rand_units(rng, m) * rng.uniform(0.0, 2 * a + 3 * t, (m, 1))
    k = m // 4
    nj[:k] = ni[:k] + 0.01 * rng.normal(size=(k, 3))
    nj[:k] /= np.linalg.norm(nj[:k], axis=1, keepdims=True)
    nj[k:k + k // 2] = ni[k:k + k // 2]
    return d, ni, nj


def one_sided(d, ni, nj, a, t):
    """(reference contacts, specification contacts, specification-only
    contacts that the reference confirms within the allowance)."""
    ref = np.array([oracle.plt_collide(d[k], ni[k], nj[k], a, t) for k in range(len(d))], dtype=np.uint8)
    got = np.array([spec.collide32(d[k], ni[k], nj[k], a, t) for k in range(len(d))], dtype=np.uint8)
    extra = np.nonzero((got == 1) & (ref == 0))[0]
    near = [spec.confirmed_by_reference(oracle, d[k], ni[k], nj[k], a, t) for k in extra]
    return ref, got, extra, near


@pytest.mark.parametrize("a,t", [(1.0, 1.0 / 199.0), (1.0, 0.1), (0.03, 0.0003)])
def test_specification_is_one_sided_on_random_pairs(a, t):
    d, ni, nj = pair_set(int(1 / t), 20000, a, t)
    ref, got, extra, near = one_sided(d, ni, nj, a, t)
    assert 0.05 < ref.mean() < 0.95
    assert np.all(got[ref == 1] == 1), "a contact of the reference is missing"
    assert all(near), "a contact only the specification reports is farther than the widening"


def test_specification_is_one_sided_near_contact():
    """Pairs placed within a few widenings of touching: stacked parallel
    disks and coplanar rims, where the widening decides."""
    rng = np.random.default_rng(9)
    a, t = 1.0, 0.005
    ds, us, vs = [], [], []
    for n in rand_units(rng, 300):
        e = np.cross(n, [1.0, 0.0, 0.0] if abs(n[0]) < 0.9 else [0.0, 1.0, 0.0])
        e /= np.linalg.norm(e)
        g = rng.uniform(-3, 3) * spec.SLACK * a
        ds.append(n * (2 * t + g) + rng.uniform(0, 1.5) * e)  # stacked, gap g from touching
        us.append(n)
        vs.append(n)
        ds.append(e * (2 * a + 2 * t + g))  # coplanar, rims g from touching
        us.append(n)
        vs.append(n)
    ref, got, extra, near = one_sided(np.array(ds), np.array(us), np.array(vs), a, t)
    assert np.all(got[ref == 1] == 1)
    assert len(extra) > 20 and all(near)


def test_reference_sweep_on_specification_equals_brute_force():
    box = (1.0, 1.2, 1.0)
    a0, t0 = 0.09, 0.01
    X0, U0 = start_config(40, np.array(box), a0, t0, 11)
    lam, c_m = 1.4, 0.04
    s = oracle.PlateletSystem(box, X0, U0, a0, t0, lam=lam, c_m=c_m, c_r=0.3, N_l=4, seed=21, sweep=2,
                              contact=spec.address())
    X, U = X0, U0
    for k in range(2):
        X, U, acc = brute_sweep(X, U, box, a0, t0, lam, c_m, 0.3, 4, 21, 2 + k, collide=spec.collide32)
        assert s.sweep() == acc
        SX, SU = s.state()
        np.testing.assert_array_equal(SX, X)
        np.testing.assert_array_equal(SU, U)


def test_budget_decided_contact_is_a_near_contact():
    """A pair whose contact the kernel reports only because an arc's
    bisection ran out of budget (found among the random thick pairs): the
    reference separates it at 2 t, and confirms contact at 2 t + 2^-12 a."""
    d, ni, nj = pair_set(10, 20000, 1.0, 0.1)
    k = 16609
    assert spec.collide32(d[k], ni[k], nj[k], 1.0, 0.1) == 1 and spec.reason(d[k], ni[k], nj[k], 1.0, 0.1) == 2
    assert oracle.plt_collide(d[k], ni[k], nj[k], 1.0, 0.1) == 0
    assert oracle.plt_collide(d[k], ni[k], nj[k], 1.0, 0.1 + 0.5 * spec.BUDGET_GAP) == 1
