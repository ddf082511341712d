"""Layout of a batch hierarchy against the meshes' own hierarchies, on the CPU.

Meshes of uneven size and depth are solved together in one hierarchy, aligned at the
finest level. Batch level D - k holds level depth_i - k of every mesh i that has one.
The host-only handles let the CPU suite check that concatenation. At every batch
level and for every mesh:
- the mesh's rows are exactly its own functions, in its own order;
- the pattern is the mesh's own, and no mesh couples with another;
- the prolongation is the mesh's own.
Rows of meshes that are smoothed at a level come first, by colour and then by mesh.
Rows of meshes whose coarsest level it is follow, mesh by mesh.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import paper_1505_03615_gb300 as L


def _meshes():
    return [
        (*meshgen.icosphere(2, 1.0, 1e-3, 1), 4),
        (*meshgen.torus_knot_tube(2, 3, 1.0, 0.12, 48, 8, 1e-6, 3), 5),
        (*meshgen.torus(1.0, 0.3, 60, 20, 1e-6, 5), 5),
        (*meshgen.ellipsoid((1.0, 0.6, 0.4), 2, 1e-6, 3), 3),
        (*meshgen.double_sheet(8, 0.05, 5, 0.5, 1e-6, 4), 5),
    ]


@pytest.fixture(scope="module")
def batch():
    meshes = _meshes()
    hb = L.lbmg_host_build_batch(meshes)
    singles = [L.lbmg_host_build(V, F, d) for V, F, d in meshes]
    yield meshes, hb, singles
    L.lbmg_host_destroy(hb)
    for h in singles:
        L.lbmg_host_destroy(h)


def _colour(corner):
    return (corner[:, 0] & 1) | ((corner[:, 1] & 1) << 1) | ((corner[:, 2] & 1) << 2)


def _levels(batch):
    """(batch level, mesh, the mesh's own level) for every mesh present at a level."""
    meshes, hb, singles = batch
    n, Ds, d0s = L.lbmg_host_instances(hb)
    B0, BD = L.lbmg_host_levels(hb)
    for dB in range(B0, BD + 1):
        for i in range(n):
            real = int(Ds[i]) - (BD - dB)
            if real >= d0s[i]:
                yield dB, i, real


def test_instances_and_depths(batch):
    meshes, hb, singles = batch
    n, Ds, d0s = L.lbmg_host_instances(hb)
    assert n == len(meshes)
    for i, (V, F, d) in enumerate(meshes):
        assert (Ds[i], d0s[i]) == (d, L.lbmg_host_levels(singles[i])[0])
    B0, BD = L.lbmg_host_levels(hb)
    assert B0 == 0 and BD == max(Ds - d0s)


def test_each_mesh_keeps_its_functions_in_its_own_order(batch):
    meshes, hb, singles = batch
    B0, BD = L.lbmg_host_levels(hb)
    for dB in range(B0, BD + 1):
        inst = L.lbmg_host_row_instances(hb, dB)
        corner, mintri = L.lbmg_host_get_dofs(hb, dB)
        present = {i for d, i, _ in _levels(batch) if d == dB}
        assert set(np.unique(inst).tolist()) == present
        for d, i, real in _levels(batch):
            if d != dB:
                continue
            rows = np.flatnonzero(inst == i)
            c1, m1 = L.lbmg_host_get_dofs(singles[i], real)
            assert np.array_equal(corner[rows], c1) and np.array_equal(mintri[rows], m1)


def test_each_mesh_keeps_its_pattern_and_meshes_never_couple(batch):
    meshes, hb, singles = batch
    for dB, i, real in _levels(batch):
        inst = L.lbmg_host_row_instances(hb, dB)
        rp, ci = L.lbmg_host_get_pattern(hb, dB)
        n = inst.size
        rows = np.repeat(np.arange(n), np.diff(rp))
        assert (inst[rows] == inst[ci]).all()
        mine = np.flatnonzero(inst == i)
        local = np.full(n, -1)
        local[mine] = np.arange(mine.size)
        sel = inst[rows] == i
        got = sp.csr_matrix((np.ones(sel.sum()), (local[rows[sel]], local[ci[sel]])), shape=(mine.size,) * 2)
        rp1, ci1 = L.lbmg_host_get_pattern(singles[i], real)
        own = sp.csr_matrix((np.ones(ci1.size), ci1, rp1), shape=(mine.size,) * 2)
        assert got.nnz == own.nnz and abs(got - own).max() == 0


def test_each_mesh_keeps_its_prolongation(batch):
    meshes, hb, singles = batch
    n, Ds, d0s = L.lbmg_host_instances(hb)
    for dB, i, real in _levels(batch):
        if real == d0s[i]:
            continue
        inst_f = L.lbmg_host_row_instances(hb, dB)
        inst_c = L.lbmg_host_row_instances(hb, dB - 1)
        local_c = np.full(inst_c.size, -1)
        mine_c = np.flatnonzero(inst_c == i)
        local_c[mine_c] = np.arange(mine_c.size)
        par, w = L.lbmg_host_get_prolongation(hb, dB)
        rows = np.flatnonzero(inst_f == i)
        p, wb = par[rows], w[rows]
        p_local = np.where(p >= 0, local_c[np.maximum(p, 0)], -1)
        assert (inst_c[p[p >= 0]] == i).all()
        p1, w1 = L.lbmg_host_get_prolongation(singles[i], real)
        assert np.array_equal(p_local, p1) and np.array_equal(wb, w1)


def test_rows_by_colour_then_mesh_and_coarsest_blocks_last(batch):
    meshes, hb, singles = batch
    n, Ds, d0s = L.lbmg_host_instances(hb)
    B0, BD = L.lbmg_host_levels(hb)
    for dB in range(B0, BD + 1):
        inst = L.lbmg_host_row_instances(hb, dB)
        corner, _ = L.lbmg_host_get_dofs(hb, dB)
        real = Ds[inst] - (BD - dB)
        smoothed = real > d0s[inst]
        ns = int(smoothed.sum())
        assert smoothed[:ns].all() and not smoothed[ns:].any()
        key = _colour(corner[:ns]).astype(np.int64) * n + inst[:ns]
        assert (np.diff(key) >= 0).all()
        assert (np.diff(inst[ns:]) >= 0).all()
