"""The seeded input generators: topology, sizes and determinism of the synthetic meshes.

The solver's inputs stand in for the paper's models (Section 5): closed surfaces of
genus 0 and 1, a thin knotted tube whose distant parts share coarse voxels, and two
parallel sheets half a finest voxel apart.  These tests check that the generators
deliver exactly those shapes and sizes, independently of the method.
"""
import numpy as np
import pytest
from scipy.sparse import coo_matrix
from scipy.sparse.csgraph import connected_components

import meshgen


def _directed_edges(F):
    return np.concatenate([F[:, [0, 1]], F[:, [1, 2]], F[:, [2, 0]]]).astype(np.int64)


def _edge_stats(V, F):
    """(undirected edge count, directed edges without a reverse, repeated directed edges)."""
    nv = V.shape[0]
    e = _directed_edges(F)
    key = e[:, 0] * nv + e[:, 1]
    rev = e[:, 1] * nv + e[:, 0]
    ukey, cnt = np.unique(key, return_counts=True)
    repeated = int((cnt > 1).sum())
    unmatched = int((~np.isin(rev, ukey)).sum())
    und = np.unique(np.minimum(key, rev))
    return und.size, unmatched, repeated


def _components(V, F):
    e = _directed_edges(F)
    g = coo_matrix((np.ones(e.shape[0]), (e[:, 0], e[:, 1])), shape=(V.shape[0],) * 2)
    return connected_components(g, directed=False)[0]


CLOSED = {
    "icosphere": (lambda: meshgen.icosphere(3), 2),
    "ellipsoid": (lambda: meshgen.ellipsoid(level=3), 2),
    "torus": (lambda: meshgen.torus(n_major=20, n_minor=8), 0),
    "knot_small": (lambda: meshgen.torus_knot_tube(n_seg=60, n_ring=12), 0),
    "knot23_200k": (lambda: meshgen.torus_knot_tube(), 0),
}


@pytest.mark.parametrize("name", sorted(CLOSED))
def test_closed_surfaces_are_oriented_manifolds_of_the_right_genus(name):
    build, chi = CLOSED[name]
    V, F = build()
    assert V.dtype == np.float64 and F.dtype == np.int32 and V.shape[1] == 3 and F.shape[1] == 3
    assert np.isfinite(V).all()
    # every vertex is used, no triangle repeats a vertex
    assert np.unique(F).size == V.shape[0]
    assert (F[:, 0] != F[:, 1]).all() and (F[:, 1] != F[:, 2]).all() and (F[:, 2] != F[:, 0]).all()
    # closed and consistently oriented: each directed edge once, its reverse present
    ne, unmatched, repeated = _edge_stats(V, F)
    assert unmatched == 0 and repeated == 0
    assert 2 * ne == 3 * F.shape[0]
    # Euler characteristic V - E + F = 2 - 2 genus, one component
    assert V.shape[0] - ne + F.shape[0] == chi
    assert _components(V, F) == 1


def test_triangle_counts_of_the_named_workloads():
    assert meshgen.icosphere(3)[1].shape[0] == 1280
    assert meshgen.icosphere(3)[0].shape[0] == 642
    for name, nt in (("knot23_200k_d8", 200_000), ("double_sheet_1m_d9", 1_000_000)):
        V, F = meshgen.CONFIGS[name]["mesh"]()
        assert F.shape[0] == nt
    # the 4M-triangle tube has the same construction: n_seg x n_ring x 2 triangles
    V, F = meshgen.torus_knot_tube(3, 5, 1.0, 0.02, 100, 20, 1e-7, 6)
    assert F.shape[0] == 100 * 20 * 2


def test_knot_tube_is_a_circular_tube_of_the_given_radius():
    """Each ring of n_ring vertices lies on a circle of radius tube_radius about its
    centroid, in the plane normal to the ring sequence's direction."""
    n_seg, n_ring, r = 400, 24, 0.05
    V, _ = meshgen.torus_knot_tube(2, 3, 1.0, r, n_seg, n_ring, jitter=0.0)
    rings = V.reshape(n_seg, n_ring, 3)
    c = rings.mean(axis=1)
    dist = np.linalg.norm(rings - c[:, None, :], axis=2)
    assert np.allclose(dist, r, rtol=1e-12, atol=1e-12)
    # distant parts of the knot never touch, yet lie within the support (two cells wide)
    # of one hat function of the depth-2 grid, where the connectivity split matters
    d = np.linalg.norm(c[:, None, :] - c[None, :, :], axis=2)
    idx = np.arange(n_seg)
    gap = np.minimum(np.abs(idx[:, None] - idx[None, :]), n_seg - np.abs(idx[:, None] - idx[None, :]))
    far = d[gap > n_seg // 8]
    assert far.min() > 4 * r
    S = 1.1 * np.ptp(V, axis=0).max()
    assert far.min() + 2 * r < 2 * S / 2 ** 2


def test_double_sheet_is_two_disconnected_sheets_half_a_finest_voxel_apart():
    n, depth = 40, 9
    V, F = meshgen.double_sheet(n=n, depth=depth, jitter=0.0)
    assert F.shape[0] == 2 * 2 * n * n
    assert _components(V, F) == 2
    ne, unmatched, repeated = _edge_stats(V, F)
    assert repeated == 0
    assert unmatched == 2 * 4 * n            # the boundary of each square
    assert V.shape[0] - ne + F.shape[0] == 2  # two discs
    half = V.shape[0] // 2
    off = V[half:] - V[:half]
    assert np.allclose(off[:, :2], 0.0, atol=0.0)
    assert np.allclose(off[:, 2], 0.5 * 1.1 / 2 ** depth, rtol=1e-12)
    # the depth-9 cube side of the metric's sheets is 1.1 x the largest extent (1.0)
    Vf, _ = meshgen.CONFIGS["double_sheet_1m_d9"]["mesh"]()
    assert abs(np.ptp(Vf, axis=0).max() - 1.0) < 1e-5


def test_generators_are_deterministic_and_seeded():
    a = meshgen.torus_knot_tube(n_seg=60, n_ring=12, seed=2)
    b = meshgen.torus_knot_tube(n_seg=60, n_ring=12, seed=2)
    c = meshgen.torus_knot_tube(n_seg=60, n_ring=12, seed=3)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1])
    V = meshgen.icosphere(3)[0]
    assert np.array_equal(meshgen.uniform_rhs(10), meshgen.uniform_rhs(10))
    assert np.array_equal(meshgen.sphere_harmonic_rhs(V), meshgen.sphere_harmonic_rhs(V))


def test_right_hand_sides():
    V = meshgen.icosphere(3)[0]
    f = meshgen.sphere_harmonic_rhs(V, noise=0.0)
    z = V[:, 2] / np.linalg.norm(V, axis=1)
    # the degree-3 Legendre polynomial: P3(1) = 1, P3(-1) = -1, odd, zero mean over the sphere
    assert f.shape == (V.shape[0], 1)
    for zz, p in ((1.0, 1.0), (-1.0, -1.0), (0.0, 0.0)):
        k = np.argmin(np.abs(z - zz))
        assert abs(f[k, 0] - p) < 0.05
    u = meshgen.uniform_rhs(100_000)
    assert u.shape == (100_000, 1) and u.min() >= -1 and u.max() <= 1 and abs(u.mean()) < 0.01
    assert np.array_equal(meshgen.coordinate_rhs(V), V)


@pytest.fixture(scope="module")
def batch():
    return meshgen.batch_mix(64)


def test_batch_of_uneven_meshes(batch):
    assert len(batch) == 64
    nts = np.array([F.shape[0] for _, F, _ in batch])
    depths = np.array([d for _, _, d in batch])
    # log-uniform sizes across the whole 10k-300k range (realised counts round to each shape's grid)
    assert nts.min() >= 10_000 and nts.max() <= 1.1 * 300_000
    assert nts.min() < 15_000 and nts.max() > 250_000
    assert 4.5e6 < nts.sum() < 6.5e6
    # finer octrees for larger meshes: depths 7, 8 and 9 all occur and never decrease with size
    assert set(depths.tolist()) == {7, 8, 9}
    o = np.argsort(nts, kind="stable")
    assert (np.diff(depths[o]) >= 0).all()
    # tori, ellipsoids and knots in turn, each closed and of its genus
    for i, (V, F, _) in enumerate(batch[:6]):
        ne, unmatched, repeated = _edge_stats(V, F)
        assert unmatched == 0 and repeated == 0
        chi = V.shape[0] - ne + F.shape[0]
        assert chi == (2 if i % 3 == 1 else 0)
