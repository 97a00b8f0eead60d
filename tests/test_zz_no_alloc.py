"""srm_certify_noalloc, the certification for callers that cannot allocate
device memory (plug-ins of a host application that owns every device
allocation, code under a fixed device-memory budget, latency-bound paths
where an allocation could block).  The call takes the caller's device
buffers and keeps its working memory in a static device array of the
library.  Here it is called through the C interface on two calls in a row
and must give exactly the results of srm_certify on the same configuration,
and of the reference's O(N^2) brute force: the same binary64 predicate on
the same values, over grids that both contain every pair closer than 2 R_max
(which holds the smallest gap in the dense and overlapping states used).
This file is collected last so that a failure here leaves every other test
already run."""
import numpy as np
import pytest

import oracle
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def _certify_both(g, w, stream):
    import torch
    x, R = g.positions()
    ref_pairs, ref_gap, _ = g.certify()
    xd = torch.from_numpy(np.ascontiguousarray(x)).cuda()
    rd = torch.from_numpy(np.ascontiguousarray(R)).cuda()
    torch.cuda.synchronize()
    out = []
    for _ in range(2):  # two calls in a row share the static working memory
        out.append(srm.srm_certify_noalloc(w.dim, w.box, w.n, xd.data_ptr(), rd.data_ptr(), stream))
    # the reference's brute force over all pairs (pair count and smallest gap)
    _, bf_pairs, bf_gap = oracle.pairs_brute(w.dim, w.box, x, R)
    assert (bf_pairs, bf_gap) == (ref_pairs, ref_gap)
    return (ref_pairs, ref_gap), out


@pytest.mark.parametrize("dim,n,phi", [(3, 3000, 0.40), (2, 4000, 0.55)])
def test_noalloc_certify_matches_certify(dim, n, phi):
    import torch
    w = srm_inputs._mono("noalloc", dim, n, phi, 0.1, 17 + dim)
    stream = torch.cuda.current_stream().cuda_stream
    g = srm.Rve(w.dim, w.box, w.radii, w.target_phi, w.seed, init="explicit", positions=w.x,
                c_m=w.c_m, c_w=0.02, stream=stream)
    assert g.run_to_target()["converged"]
    # dense clean state: no pairs, smallest gap positive
    ref, out = _certify_both(g, w, stream)
    assert ref[0] == 0 and ref[1] > 0
    for pairs, gap in out:
        assert pairs == ref[0] and gap == ref[1]
    # swollen state with overlaps: pair count and (negative) smallest gap
    g.set_scale(g.state()["lambda"] * 1.03)
    ref, out = _certify_both(g, w, stream)
    assert ref[0] > 0 and ref[1] < 0
    for pairs, gap in out:
        assert pairs == ref[0] and gap == ref[1]
    g.close()


def test_noalloc_rejects_beyond_maximum():
    import torch
    n = 32769  # one more than SRM_NOALLOC_MAX_PARTICLES
    xd = torch.zeros(n * 3, dtype=torch.float64, device="cuda")
    rd = torch.full((n,), 1e-3, dtype=torch.float64, device="cuda")
    with pytest.raises(srm.SrmError) as e:
        srm.srm_certify_noalloc(3, (1.0, 1.0, 1.0), n, xd.data_ptr(), rd.data_ptr())
    assert e.value.status == 1 and "SRM_NOALLOC_MAX_PARTICLES" in e.value.message


def test_noalloc_rejects_nan_radius():
    import torch
    w = srm_inputs._mono("noalloc_nan", 3, 500, 0.35, 0.3, 23)  # dense RSA state at 0.3
    x = torch.from_numpy(np.ascontiguousarray(w.x)).cuda()
    r = np.ascontiguousarray(w.radii * 1.0)
    r[17] = np.nan
    rd = torch.from_numpy(r).cuda()
    with pytest.raises(srm.SrmError) as e:
        srm.srm_certify_noalloc(3, w.box, w.n, x.data_ptr(), rd.data_ptr())
    assert e.value.status == 1 and "finite" in e.value.message
    # a valid call right after it works on the same static memory
    r[17] = r[16]
    rd = torch.from_numpy(r).cuda()
    pairs, gap = srm.srm_certify_noalloc(3, w.box, w.n, x.data_ptr(), rd.data_ptr())
    assert (pairs, gap) == oracle.pairs_brute(3, w.box, w.x, r)[1:]
