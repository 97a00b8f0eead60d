"""Batches, serving slots and checkpoints through the C interface.

Every RVE keeps its own state, grid, buffers and counter-based draws, so its
result must not depend on which other RVEs share the launches: the tests
compare each member of a batch (and each job admitted into a running
serving batch) with the same job run alone, bit for bit, in both
precisions; FP64 members are also compared with the FP64 reference.  A
checkpointed handle must continue exactly as the original."""
import numpy as np
import pytest

import oracle
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def mixed_workloads():
    ws = [srm_inputs._mono("b0", 2, 700, 0.45, 0.1, 31),
          srm_inputs._mono("b1", 3, 1500, 0.35, 0.1, 32),
          srm_inputs._mono("b2", 2, 2300, 0.50, 0.1, 33),
          srm_inputs._mono("b3", 3, 400, 0.40, 0.1, 34),
          srm_inputs._mono("b4", 3, 3100, 0.30, 0.1, 35)]
    return ws


def job_of(w, precision):
    return srm.make_job(w.dim, w.box, w.radii, w.target_phi, w.seed, c_m=w.c_m, c_w=0.02,
                        precision=precision, init="explicit", positions=w.x)


def alone(w, precision):
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, c_m=w.c_m, c_w=0.02,
                precision=precision, init="explicit", positions=w.x)
    assert g.run_to_target()["converged"]
    x, r = g.positions()
    st = g.state()
    g.close()
    return x, r, st


@pytest.mark.parametrize("precision", [64, 32])
def test_batch_members_equal_alone(precision):
    ws = mixed_workloads()
    b = srm.Batch([job_of(w, precision) for w in ws])
    assert b.run()
    for i, w in enumerate(ws):
        x, r, st = alone(w, precision)
        xb, rb = b.positions(i)
        np.testing.assert_array_equal(xb, x)
        np.testing.assert_array_equal(rb, r)
        sb = b.state(i)
        assert sb["sweeps"] == st["sweeps"] and sb["iterations"] == st["iterations"]
        pairs, gap, phi = b.certify(i)
        assert pairs == 0 and abs(phi - w.target_phi) < 1e-9
        if precision == 64:
            o = oracle.System(w.dim, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=0.02,
                              c_m=w.c_m, seed=w.seed)
            o.run()
            np.testing.assert_array_equal(xb, o.x)
    b.close()


@pytest.mark.parametrize("precision", [32, 64])
def test_serving_slots_admit_while_running(precision):
    """Jobs admitted at different times into a running batch (continuous
    batching) give the results they give alone."""
    ws = mixed_workloads()
    b = srm.Batch(slots=3, max_particles=4000, max_cells=400000, precision=precision)
    queue = list(range(len(ws)))
    running, done = {}, {}
    free = [0, 1, 2]
    steps = 0
    while queue or running:
        while queue and free:
            k = queue.pop(0)
            s = free.pop(0)
            b.admit(s, job_of(ws[k], precision))
            running[s] = k
        b.advance(8)
        steps += 1
        for s in b.poll():
            k = running.pop(s)
            done[k] = b.positions(s)
            b.release(s)
            free.append(s)
        assert steps < 20000
    for k, w in enumerate(ws):
        x, r, _ = alone(w, precision)
        np.testing.assert_array_equal(done[k][0], x)
        np.testing.assert_array_equal(done[k][1], r)
    b.close()


def test_slot_rejects_oversized_job():
    w = srm_inputs._mono("big", 3, 3000, 0.3, 0.1, 5)
    b = srm.Batch(slots=1, max_particles=1000, max_cells=1000, precision=32)
    with pytest.raises(srm.SrmError) as e:
        b.admit(0, job_of(w, 32))
    assert e.value.status == 1
    b.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_checkpoint_resume_bit_exact(precision):
    w = srm_inputs._mono("ck", 3, 2500, 0.42, 0.1, 41)
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, c_m=w.c_m, c_w=0.02,
                precision=precision, init="explicit", positions=w.x)
    g.run_to_target(15)
    blob = g.save()
    g.run_to_target(15)
    xa, ra = g.positions()
    sa = g.state()
    h = srm.srm_load(blob)
    st = h.state()
    assert st["iterations"] == 15 and st["precision"] == precision
    h.run_to_target(15)
    xb, rb = h.positions()
    sb = h.state()
    np.testing.assert_array_equal(xa, xb)
    np.testing.assert_array_equal(ra, rb)
    assert sa["sweep"] == sb["sweep"] and sa["lambda"] == sb["lambda"]
    g.close()
    h.close()


@pytest.mark.parametrize("precision", [64, 32])
def test_launch_shape_does_not_change_results(precision):
    """The autotuner and explicit launch shapes (one sweep block per SM, the
    smallest staging capacity, which sends dense cells down the overflow
    path) change the speed only: every member ends bit for bit as alone."""
    ws = mixed_workloads()
    b = srm.Batch([job_of(w, precision) for w in ws])
    t = b.autotune(8)
    assert t["candidates"] >= 2 and t["ns_per_particle_sweep"] > 0
    assert b.tuning()["stage_capacity"] == t["stage_capacity"]
    assert b.run(3) in (True, False)  # every RVE is between iterations after tuning
    b.set_tuning(1, 64)
    tn = b.tuning()
    assert tn["sweep_blocks_per_sm"] == 1 and tn["stage_capacity"] == 64
    b.advance(24)
    b.set_tuning(0, 0)
    assert b.run()
    for i, w in enumerate(ws):
        x, r, st = alone(w, precision)
        xb, _ = b.positions(i)
        np.testing.assert_array_equal(xb, x)
        assert b.state(i)["sweeps"] == st["sweeps"]
    b.close()


def test_slots_of_one_dimension():
    """A pool of 2D slots (one sweep launch per super-step) runs 2D jobs as
    alone and rejects a 3D job."""
    ws = [w for w in mixed_workloads() if w.dim == 2]
    b = srm.Batch(slots=2, max_particles=4000, max_cells=400000, dim=2, precision=32)
    w3 = [w for w in mixed_workloads() if w.dim == 3][0]
    with pytest.raises(srm.SrmError) as e:
        b.admit(0, job_of(w3, 32))
    assert e.value.status == 1
    for s, w in enumerate(ws):
        b.admit(s, job_of(w, 32))
    steps, finished = 0, set()
    while len(finished) < len(ws) and steps < 20000:
        b.advance(8)
        finished.update(b.poll())
        steps += 1
    for s, w in enumerate(ws):
        x, r, _ = alone(w, 32)
        np.testing.assert_array_equal(b.positions(s)[0], x)
    b.close()
