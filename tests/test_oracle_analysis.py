"""Pins of the reference structure descriptors (Section 3.2: nearest-neighbour
distances, Fig. 4d; local volume fraction from Voronoi cells, Figs. 5 and 7;
radial distribution of the centres) against closed forms on lattices and
against independent library implementations (scipy's periodic KD-tree,
numpy histograms)."""
import math

import numpy as np
import pytest

import oracle

scipy_spatial = pytest.importorskip("scipy.spatial")


def lattice(dim, n, a):
    """Simple square / cubic lattice of n per axis, spacing a, points at
    cell centres ((i + 0.5) a)."""
    g = (np.arange(n) + 0.5) * a
    if dim == 2:
        return np.stack(np.meshgrid(g, g, indexing="ij"), axis=-1).reshape(-1, 2)
    return np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)


@pytest.mark.parametrize("dim", [2, 3])
def test_nn_lattice_closed_form(dim):
    n, a, R = 6, 0.25, 0.1
    X = lattice(dim, n, a)
    d, j, g = oracle.nn(dim, (n * a,) * dim, X, np.full(len(X), R))
    np.testing.assert_allclose(d, a, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g, a - 2 * R, rtol=0, atol=1e-15)


@pytest.mark.parametrize("dim", [2, 3])
def test_nn_against_periodic_kdtree(dim):
    rng = np.random.default_rng(3 + dim)
    box = np.array([1.0, 0.8, 1.3][:dim])
    X = rng.random((400, dim)) * box
    R = rng.uniform(0.005, 0.02, 400)
    d, j, g = oracle.nn(dim, box, X, R)
    tree = scipy_spatial.cKDTree(X, boxsize=box)
    dd, jj = tree.query(X, k=2)
    np.testing.assert_allclose(d, dd[:, 1], rtol=1e-13)
    np.testing.assert_array_equal(j, jj[:, 1])
    # smallest surface gap: against all pairs from the tree within a cutoff
    pairs = tree.query_pairs(0.5, output_type="ndarray")
    diff = X[pairs[:, 0]] - X[pairs[:, 1]]
    diff -= np.round(diff / box) * box
    gp = np.sqrt((diff ** 2).sum(1)) - R[pairs[:, 0]] - R[pairs[:, 1]]
    ref = np.full(len(X), np.inf)
    np.minimum.at(ref, pairs[:, 0], gp)
    np.minimum.at(ref, pairs[:, 1], gp)
    np.testing.assert_allclose(g, ref, rtol=1e-12, atol=1e-15)


def test_rdf_cubic_lattice_shells():
    # 8^3 points, spacing a: 6 neighbours at a, 12 at sqrt(2) a, 8 at sqrt(3) a, 6 at 2 a
    n, a = 8, 0.125
    X = lattice(3, n, a)
    N = len(X)
    c, g = oracle.rdf(3, (1.0, 1.0, 1.0), X, 2.2 * a, 22)
    expect = {10: 6, 14: 12, 17: 8, 20: 6}  # bin = floor(S / (0.1 a))
    for b in range(22):
        assert c[b] == N * expect.get(b, 0), (b, c[b])


@pytest.mark.parametrize("dim", [2, 3])
def test_rdf_against_numpy_histogram(dim):
    rng = np.random.default_rng(11 + dim)
    box = np.ones(dim)
    X = rng.random((600, dim))
    r_max, bins = 0.3, 30
    c, g = oracle.rdf(dim, box, X, r_max, bins)
    tree = scipy_spatial.cKDTree(X, boxsize=box)
    pairs = tree.query_pairs(r_max, output_type="ndarray")
    diff = X[pairs[:, 0]] - X[pairs[:, 1]]
    diff -= np.round(diff / box) * box
    S = np.sqrt((diff ** 2).sum(1))
    ref, _ = np.histogram(S, bins=bins, range=(0.0, r_max))
    np.testing.assert_array_equal(c, 2 * ref)
    # uniform points: g close to 1 away from the first bins (Poisson noise)
    assert abs(np.mean(g[5:]) - 1.0) < 0.05


@pytest.mark.parametrize("dim,k", [(2, 3), (3, 3), (2, 5)])
def test_voronoi_lattice_closed_form(dim, k):
    # k (odd) voxels per lattice cell and axis: voxel centres never tie, every
    # Voronoi cell is the lattice cell, LVF = v / a^d exactly (to rounding)
    n, a, R = 5, 0.2, 0.07
    X = lattice(dim, n, a)
    cnt, lvf = oracle.voronoi_lvf(dim, (n * a,) * dim, X, np.full(len(X), R), (k * n,) * dim)
    assert np.all(cnt == k ** dim)
    v = math.pi * R * R if dim == 2 else 4.0 / 3.0 * math.pi * R ** 3
    np.testing.assert_allclose(lvf, v / a ** dim, rtol=1e-13)


@pytest.mark.parametrize("dim", [2, 3])
def test_voronoi_against_periodic_kdtree(dim):
    rng = np.random.default_rng(21 + dim)
    box = np.array([1.0, 0.75, 1.2][:dim])
    N = 150
    X = rng.random((N, dim)) * box
    R = rng.uniform(0.01, 0.03, N)
    M = np.array([40, 30, 48][:dim])
    cnt, lvf = oracle.voronoi_lvf(dim, box, X, R, M)
    assert cnt.sum() == np.prod(M)
    axes = [(np.arange(M[a]) + 0.5) * (box[a] / M[a]) for a in range(dim)]
    C = np.stack(np.meshgrid(*axes, indexing="ij"), axis=-1).reshape(-1, dim)
    _, owner = scipy_spatial.cKDTree(X, boxsize=box).query(C)
    np.testing.assert_array_equal(cnt, np.bincount(owner, minlength=N))
    v = math.pi * R ** 2 if dim == 2 else 4.0 / 3.0 * math.pi * R ** 3
    np.testing.assert_allclose(lvf, v / (cnt * np.prod(box / M)), rtol=1e-13)
