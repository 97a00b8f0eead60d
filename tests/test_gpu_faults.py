"""Failure paths on the GPU without faulting it: the one-launch sweep waits
for neighbouring cells with a bounded number of polls; with wait_limit < 0
every such wait gives up at once (as if it waited on a flag that nothing
sets), the RVE reports SRM_E_DEVICE_TIMEOUT through its status word, the
kernel returns, and the context stays usable."""
import numpy as np
import pytest

import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("precision", [32, 64])
def test_bounded_wait_reports_timeout(precision):
    w = srm_inputs._mono("t", 3, 3000, 0.4, 0.1, 3)
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                c_m=w.c_m, precision=precision, wait_limit=-1)
    with pytest.raises(srm.SrmError) as e:
        g.step()
    assert e.value.status == 5
    g.close()
    # a fresh handle on the same context works
    h = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                c_m=w.c_m, precision=precision)
    assert h.run_to_target()["converged"] and h.certify()[0] == 0
    h.close()


def test_iteration_cap_reports_not_converged():
    w = srm_inputs._mono("t", 2, 2000, 0.5, 0.1, 4)
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                c_m=w.c_m)
    info = g.run_to_target(5)
    assert not info["converged"] and info["iterations"] == 5
    info = g.run_to_target()
    assert info["converged"]
    g.close()


def test_try_count_beyond_counter_field_rejected():
    """The try index l takes 16 bits of the generator's counter word, so
    N_l above 65535 is refused at initialisation with SRM_E_ARG; 65535 is
    accepted."""
    w = srm_inputs._mono("t", 2, 500, 0.3, 0.1, 5)
    with pytest.raises(srm.SrmError) as e:
        srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x, c_m=w.c_m,
                N_l=65536)
    assert e.value.status == 1
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x, c_m=w.c_m,
                N_l=65535)
    g.close()
