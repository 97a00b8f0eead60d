"""Image-particle periodicity (Section 2: the alternative to the minimum
image of Alg 5) on the GPU through the C interface, against the reference's
images mode (entries x + s L kept move by move, tests/test_oracle_images.py).

FP64 form: every iteration, full run and pair list equals the reference's
images mode bit for bit, and the minimum-image run bit for bit too (only a
pair within rounding of contact could tell the two apart).  FP32 form: its
cell-relative offsets already place every candidate at its image beside the
home cell, so the flag changes nothing.  Platelets: the images mode of the
kernel equals the reference's on the kernel specification's contact
predicate, bit for bit."""
import numpy as np
import pytest

import oracle
import plt_kernel_spec as spec
import srm_inputs
import paper_2605_18254_gb300 as srm
from test_gpu_parity import assert_same_state, pair, small_3d
from test_oracle_images import brute_images, crowded

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("maker", [lambda: srm_inputs.disks_1k(seed=6, n=800),
                                   lambda: small_3d(2000, 0.45, seed=8)])
def test_fp64_iterations_equal_reference_images_mode(maker):
    w = maker()
    g, o = pair(w, images=True)
    gm, om = pair(w)  # minimum image, for the cross-check
    for _ in range(10):
        gi = g.step()
        acc, oi = o.iterate()
        assert gi["result"] == acc and gi["k_sweeps"] == oi["k_sweeps"]
        assert_same_state(g, o)
        gm.step()
    np.testing.assert_array_equal(g.positions()[0], gm.positions()[0])


def test_fp64_full_run_equals_reference_images_mode():
    w = small_3d(1500, 0.40, seed=9)
    g, o = pair(w, images=True)
    info = g.run_to_target()
    o.run()
    assert info["converged"]
    assert_same_state(g, o)
    c = o.counters()
    assert info["sweeps"] == c["sweeps"] and info["accepted"] == c["accepted"]
    pairs, gap, phi = g.certify()
    assert pairs == 0 and gap > 0 and abs(phi - w.target_phi) < 1e-9
    assert o.pairs().shape == (0, 2)


@pytest.mark.parametrize("dim,n,seed", [(2, 900, 1), (3, 700, 2)])
def test_pair_lists_equal_explicit_copies(dim, n, seed):
    """Overlapping configurations crowded against the faces: the GPU's pair
    list in images mode equals the reference's and a brute force over
    explicit periodic copies."""
    box, x, r = crowded(dim, n, seed)
    w = srm_inputs.Workload("crowded", dim, box, r, x, 0.3, seed, c_m=0.1 * float(np.mean(r)))
    # the crowded set overlaps: start at a scale where it does not, then swell
    g = srm.Rve(dim, box, r, 0.3, seed, init="explicit", positions=x, precision=64, c_m=w.c_m, lambda0=1e-3,
                images=True)
    g.set_scale(1.0)
    got = [tuple(p) for p in g.overlap_pairs().tolist()]
    o = oracle.System(dim, box, x, r, images=True)
    assert got == [tuple(p) for p in o.pairs().tolist()] == brute_images(dim, box, x, r)
    assert len(got) > 20
    g.close()


def test_fp32_form_unchanged_by_the_flag():
    w = small_3d(3000, 0.45, seed=10)
    runs = []
    for images in (False, True):
        g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x, precision=32,
                    c_m=w.c_m, c_w=w.c_w, images=images)
        g.run_to_target(15)
        runs.append(g.positions()[0])
        g.close()
    np.testing.assert_array_equal(runs[0], runs[1])


@pytest.mark.parametrize("kernel", [0, 1])
def test_platelet_sweeps_equal_reference_images_mode(kernel):
    """Both platelet sweep kernels (a block per cell with the staged
    neighbourhood; a warp per cell)."""
    w = srm_inputs.platelets(seed=11, n=3000, aspect=20.0, rho_t=3.0)
    lam = 2.5 * w.lambda0
    args = dict(c_w=w.c_w, c_m=0.05 * w.extra["D"], c_r=0.05)
    g = srm.Platelets(w.box, w.x, w.u, w.a0, w.t0, lam, 1.0, w.seed, images=True, sweep_kernel=kernel, **args)
    o = oracle.PlateletSystem(w.box, w.x, w.u, w.a0, w.t0, lam=lam, lam_t=1.0, seed=w.seed, contact=spec.address(),
                              images=True, **args)
    for _ in range(3):
        assert g.sweeps(1) == o.sweep()
        gx, gu, info = g.state()
        ox, ou = o.state()
        np.testing.assert_array_equal(gx, ox)
        np.testing.assert_array_equal(gu, ou)
        assert o.images_verify() == 0
    st = g.sweep_stats()
    assert st["staged_sweeps" if kernel == 0 else "warp_sweeps"] == 3
    g.close()
