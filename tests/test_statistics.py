"""Statistical agreement of full runs (which diverge chaotically, so they are
compared in distribution): two-sample Kolmogorov-Smirnov tests on the
nearest-neighbour surface gaps and on the pair distances below three radii
(a sample of the radial distribution), with disjoint seeds on both sides.

* CPU: the reference in canonical (coloured) order against the reference in
  plain id order (Algorithm 3 as printed): the reading of the particle order
  must not change the statistics of the result.
* GPU: the FP32 cell-relative form against the FP64 reference.
"""
import numpy as np
import pytest
from scipy import stats

import oracle
import srm_inputs

N, PHI, RVES = 400, 0.5, 16


def gaps_and_distances(x, R, box, rng, per_rve=64):
    box = np.asarray(box, dtype=float)
    d = x[:, None, :] - x[None, :, :]
    d = d - np.round(d / box) * box
    S = np.sqrt(np.sum(d * d, axis=2))
    np.fill_diagonal(S, np.inf)
    gap = S - (R[:, None] + R[None, :])
    nn = np.min(gap, axis=1) / np.mean(R)
    iu = np.triu_indices(len(x), 1)
    pd = S[iu]
    pd = pd[pd < 3.0 * np.mean(R)] / np.mean(R)
    # a subsample per RVE weakens the correlation inside one RVE
    return (rng.choice(nn, size=min(per_rve, nn.size), replace=False),
            rng.choice(pd, size=min(4 * per_rve, pd.size), replace=False))


def oracle_ensemble(seeds, literal=False):
    rng = np.random.default_rng(7 if literal else 8)
    g, p = [], []
    for s in seeds:
        w = srm_inputs._mono("ks", 2, N, PHI, 0.1, s)
        o = oracle.System(2, w.box, w.x, w.radii, lam=1.0, target_phi=PHI, c_w=0.02, c_m=w.c_m,
                          seed=s, literal=literal)
        o.run()
        assert abs(o.phi() - PHI) < 1e-9
        a, b = gaps_and_distances(o.x, o.radii(), w.box, rng)
        g.append(a)
        p.append(b)
    return np.concatenate(g), np.concatenate(p)


def test_canonical_and_literal_order_agree():
    g1, p1 = oracle_ensemble(range(1, 1 + RVES))
    g2, p2 = oracle_ensemble(range(501, 501 + RVES), literal=True)
    assert stats.ks_2samp(g1, g2).pvalue > 0.01
    assert stats.ks_2samp(p1, p2).pvalue > 0.01
    assert np.min(g1) > 0 and np.min(g2) > 0


@pytest.mark.gpu
def test_fp32_gpu_agrees_with_reference():
    import paper_2605_18254_gb300 as srm
    rng = np.random.default_rng(9)
    g, p = [], []
    for s in range(1, 1 + RVES):
        w = srm_inputs._mono("ks", 2, N, PHI, 0.1, s)
        r = srm.Rve(2, w.box, w.radii, PHI, s, c_m=w.c_m, c_w=0.02, precision=32, init="explicit",
                    positions=w.x)
        assert r.run_to_target()["converged"]
        x, R = r.positions()
        assert r.certify()[0] == 0
        a, b = gaps_and_distances(x, R, w.box, rng)
        g.append(a)
        p.append(b)
        r.close()
    g1, p1 = np.concatenate(g), np.concatenate(p)
    g2, p2 = oracle_ensemble(range(1001, 1001 + RVES))
    assert stats.ks_2samp(g1, g2).pvalue > 0.01
    assert stats.ks_2samp(p1, p2).pvalue > 0.01


# ---------------------------------------------------------------------------
# 3D: monodisperse spheres (FP32 and FP64 forms) and the benchmark's own
# input -- log-normal radii, Gaussian clusters -- at small size, each a GPU
# ensemble against a reference ensemble with disjoint seeds.
# ---------------------------------------------------------------------------
RVES3 = 12


def mono3(seed):
    return srm_inputs._mono("ks3", 3, 600, 0.40, 0.1, seed)


def poly3(seed):
    # 1500 spheres of the benchmark recipe, 6 clusters of 250
    return srm_inputs.poly_1m(seed=seed, n=1500, clusters=6)


CASES3 = {"mono_fp32": (mono3, 32), "mono_fp64": (mono3, 64), "poly_clustered_fp32": (poly3, 32)}


def oracle_ensemble3(maker, seeds, rng):
    g, p = [], []
    for s in seeds:
        w = maker(s)
        o = oracle.System(3, w.box, w.x, w.radii, lam=1.0, target_phi=w.target_phi, c_w=0.02, c_m=w.c_m, seed=s)
        o.run()
        assert abs(o.phi() - w.target_phi) < 1e-9
        a, b = gaps_and_distances(o.x, o.radii(), w.box, rng)
        g.append(a)
        p.append(b)
    return np.concatenate(g), np.concatenate(p)


@pytest.mark.gpu
@pytest.mark.parametrize("case", sorted(CASES3))
def test_3d_gpu_agrees_with_reference(case):
    import paper_2605_18254_gb300 as srm
    maker, prec = CASES3[case]
    rng = np.random.default_rng(10)
    g, p = [], []
    for s in range(1, 1 + RVES3):
        w = maker(s)
        r = srm.Rve(3, w.box, w.radii, w.target_phi, s, c_m=w.c_m, c_w=0.02, precision=prec, init="explicit",
                    positions=w.x)
        assert r.run_to_target()["converged"]
        x, R = r.positions()
        assert r.certify()[0] == 0
        a, b = gaps_and_distances(x, R, w.box, rng)
        g.append(a)
        p.append(b)
        r.close()
    g1, p1 = np.concatenate(g), np.concatenate(p)
    g2, p2 = oracle_ensemble3(maker, range(2001, 2001 + RVES3), np.random.default_rng(11))
    assert np.min(g1) > 0 and np.min(g2) > 0
    assert stats.ks_2samp(g1, g2).pvalue > 0.01, case
    assert stats.ks_2samp(p1, p2).pvalue > 0.01, case
