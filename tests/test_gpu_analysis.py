"""Structure descriptors of Section 3.2 on the GPU (through the C interface)
against the reference, on seeded synthetic configurations loaded as P at
scale 1: nearest neighbours, radial distribution and the discrete Voronoi
local volume fraction.  The FP64 form holds the input positions exactly, so
its descriptors must equal the reference bit for bit; the FP32 form stores
cell-relative binary32 offsets, so its descriptors are compared within the
rounding of the positions."""
import math

import numpy as np
import pytest

import oracle
import srm_inputs
import paper_2605_18254_gb300 as srm

pytestmark = pytest.mark.gpu


def config(dim, n, phi, seed, poly=False, clusters=0):
    """Seeded RSA configuration at volume fraction phi in a unit box."""
    if poly:
        r = srm_inputs.radii_lognormal(n, 1.0, 0.2, 0.5, 2.0, seed)
    else:
        r = np.ones(n)
    v = math.pi * np.sum(r ** 2) if dim == 2 else 4.0 / 3.0 * math.pi * np.sum(r ** 3)
    r = r * (phi / v) ** (1.0 / dim)
    box = (1.0,) * dim
    x = srm_inputs.rsa(dim, box, r, seed, clusters=clusters, sigma=5 * float(np.mean(r)) if clusters else 0.0)
    return box, x, r


def rve(dim, box, x, r, precision=64):
    return srm.Rve(dim, box, r, 0.6 if dim == 3 else 0.8, 7, c_m=0.1 * float(np.mean(r)), precision=precision,
                   init="explicit", positions=x)


CASES = [
    (2, 3000, 0.30, 1, True, 0),
    (3, 2000, 0.25, 2, False, 0),
    (3, 2500, 0.10, 3, True, 25),   # clustered, sparse regions: multi-ring searches
    (2, 40, 0.20, 4, False, 0),     # three cells per axis: searches cover the whole grid
]


@pytest.mark.parametrize("dim,n,phi,seed,poly,clusters", CASES)
def test_nearest_bit_exact(dim, n, phi, seed, poly, clusters):
    box, x, r = config(dim, n, phi, seed, poly, clusters)
    g = rve(dim, box, x, r)
    d, j, gap = g.nearest()
    g.close()
    od, oj, og = oracle.nn(dim, box, x, r)
    np.testing.assert_array_equal(d, od)
    np.testing.assert_array_equal(j, oj)
    np.testing.assert_array_equal(gap, og)


@pytest.mark.parametrize("dim,n,phi,seed,poly,clusters", CASES)
def test_rdf_bit_exact(dim, n, phi, seed, poly, clusters):
    box, x, r = config(dim, n, phi, seed, poly, clusters)
    g = rve(dim, box, x, r)
    for r_max, bins in ((6 * float(np.mean(r)), 60), (0.5, 100)):
        c, gr = g.rdf(r_max, bins)
        oc, og = oracle.rdf(dim, box, x, r_max, bins)
        np.testing.assert_array_equal(c, oc)
        np.testing.assert_array_equal(gr, og)
    with pytest.raises(srm.SrmError):
        g.rdf(0.51, 10)
    g.close()


@pytest.mark.parametrize("dim,n,phi,seed,poly,clusters", CASES)
def test_voronoi_bit_exact(dim, n, phi, seed, poly, clusters):
    box, x, r = config(dim, n, phi, seed, poly, clusters)
    M = (300, 300) if dim == 2 else (48, 48, 48)
    g = rve(dim, box, x, r)
    c, lvf = g.voronoi_lvf(M)
    g.close()
    oc, olvf = oracle.voronoi_lvf(dim, box, x, r, M)
    assert c.sum() == np.prod(M)
    np.testing.assert_array_equal(c, oc)
    np.testing.assert_array_equal(lvf, olvf)


def test_fp32_form_close():
    box, x, r = config(3, 2000, 0.2, 5, True, 0)
    g = rve(3, box, x, r, precision=32)
    d, j, gap = g.nearest()
    c, lvf = g.voronoi_lvf((40, 40, 40))
    cnt, gr = g.rdf(0.1, 50)
    g.close()
    od, oj, og = oracle.nn(3, box, x, r)
    np.testing.assert_allclose(d, od, rtol=1e-6)
    np.testing.assert_allclose(gap, og, atol=1e-6)
    assert np.mean(j == oj) > 0.999
    oc, _ = oracle.voronoi_lvf(3, box, x, r, (40, 40, 40))
    assert np.abs(c - oc).sum() <= 0.001 * c.sum()
    occ, _ = oracle.rdf(3, box, x, 0.1, 50)
    assert np.abs(cnt - occ).sum() <= 0.001 * occ.sum()


def regime_lvf_std(c_w, c_m_rel, seed):
    n, phi = 2000, 0.5
    r_t = math.sqrt(phi / (n * math.pi))
    g = srm.Rve(2, (1.0, 1.0), ("mono", r_t * (0.1 / phi) ** 0.5), phi, seed, n=n, c_m=c_m_rel * r_t, c_w=c_w,
                precision=32, init="rsa", f0=0.1)
    assert g.run_to_target(20000)["converged"]
    assert g.certify()[0] == 0
    c, lvf = g.voronoi_lvf((200, 200))
    g.close()
    return float(np.std(lvf))


def test_clustered_regime_broadens_lvf():
    """Fast swelling with short migration leaves clusters (Section 3.2, Fig.
    5): at the same volume fraction the spread of the local volume fraction
    is clearly larger than after slow swelling with long migration."""
    eq = np.mean([regime_lvf_std(0.002, 0.5, s) for s in (1, 2)])
    cl = np.mean([regime_lvf_std(0.01, 0.03, s) for s in (1, 2)])
    assert cl > 1.4 * eq, (cl, eq)
