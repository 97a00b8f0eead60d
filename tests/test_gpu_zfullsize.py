"""The benchmark workload at full size (1e6 polydisperse clustered spheres,
FP32 form, the launch configuration bench.py times), generated to its
target through the C interface; the reference checks what holds at any size:
its own cell-list certification finds no overlapping pair in the final
state, the volume fraction is the target, and every particle is in the
box."""
import numpy as np
import pytest

import oracle
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def test_poly_1m_to_target_certified_by_the_reference():
    w = srm_inputs.poly_1m()
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x, precision=32,
                c_m=w.c_m, c_w=w.c_w, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake)
    info = g.run_to_target()
    assert info["converged"]
    pairs, gap, phi = g.certify()
    assert pairs == 0 and gap > 0 and abs(phi - w.target_phi) < 1e-9
    x, R = g.positions()
    g.close()
    assert x.shape == (w.n, 3) and np.all(x >= 0.0) and np.all(x < np.asarray(w.box))
    cnt, min_gap = oracle.certify(w.dim, w.box, x, R)
    assert cnt == 0 and min_gap > 0
    vol = 4.0 / 3.0 * np.pi * np.sum(R ** 3) / np.prod(w.box)
    assert vol == pytest.approx(w.target_phi, rel=1e-9)


@pytest.mark.parametrize("iters", [0, 300])
def test_poly_1m_one_sweep_fp32_against_reference(iters):
    """One sweep of the FP32 form at full size (1e6 spheres) against the
    FP64 reference's sweep from the same state: at the clustered start
    (swollen by 1%), and at the state the GPU run reaches after `iters`
    iterations (exported through srm_positions and imported into both).
    Every particle within 1e-5 of the mean radius, except groups linked to
    decisions the reference took within 1e-5 of contact (test_gpu_parity's
    fp32_sweep_check)."""
    from test_gpu_parity import fp32_sweep_check
    w = srm_inputs.poly_1m()
    lam = 1.0
    if iters:
        g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x, precision=32,
                    c_m=w.c_m, c_w=w.c_w, N_k=w.N_k, N_l=w.N_l, N_shake=w.N_shake)
        g.run_to_target(iters)
        lam = g.state()["lambda"]
        x, _ = g.positions()
        g.close()
        w = srm_inputs.Workload(w.name, w.dim, w.box, w.radii, x, w.target_phi, w.seed, c_m=w.c_m)
    frac, bad, roots = fp32_sweep_check(w, lam * 1.01, w.c_m)
    print(f"iters {iters}: lambda {lam:.6f}, out of tolerance {bad}, near-contact decisions {roots}")
    assert frac > 0.9999
