"""Steps of the hierarchy build on the GPU (options.gpu_clip = 1), against the host builder:
the triangles cut into finest-voxel pieces (row a1, one thread per triangle) and, on every
level, the sorted (corner, triangle) pairs and the split labelling of each corner's support
into connected components (row a2, one thread per corner).

The build from the GPU's pieces and labels must give the same split functions, patterns and
prolongation as the host's, exactly; the matrices assembled from the two agree to 1e-13 of
their largest entry (the pieces' vertices differ at most by FMA contraction in the plane
intersections, a few units of the last place).  The seeded meshes include nearly touching
sheets (heavy splitting) and a (3,5) knot on the bench's depth-10 grid."""
import time

import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

MESHES = {
    "sphere": lambda: (*meshgen.icosphere(3, 1.0, 1e-3, 1), 5),
    "knot": lambda: (*meshgen.torus_knot_tube(2, 3, 1.0, 0.04, 400, 40, 1e-6, 2), 7),
    "sheets": lambda: (*meshgen.double_sheet(60, 0.05, 6, 0.5, 1e-6, 4), 7),
    "knot35_d10": lambda: (*meshgen.torus_knot_tube(3, 5, 1.0, 0.02, 1000, 40, 1e-6, 3), 10),
}


@pytest.mark.parametrize("mesh", list(MESHES))
def test_gpu_pieces_give_the_host_builders_hierarchy(mesh):
    V, F, depth = MESHES[mesh]()
    t0 = time.perf_counter()
    hc = L.lbmg_host_build(V, F, depth)
    t1 = time.perf_counter()
    hg = L.lbmg_host_build(V, F, depth, gpu_clip=1)
    t2 = time.perf_counter()
    try:
        print(f"\n{mesh}: host build {t1 - t0:.2f} s on the host cores, {t2 - t1:.2f} s with the GPU steps")
        assert L.lbmg_host_levels(hc) == L.lbmg_host_levels(hg)
        d0, D = L.lbmg_host_levels(hc)
        for d in range(d0, D + 1):
            assert L.lbmg_host_level_info(hc, d) == L.lbmg_host_level_info(hg, d), d
            for get in (L.lbmg_host_get_dofs, L.lbmg_host_get_pattern):
                for a, b in zip(get(hc, d), get(hg, d)):
                    assert np.array_equal(a, b), (d, get.__name__)
            if d > d0:
                for a, b in zip(L.lbmg_host_get_prolongation(hc, d), L.lbmg_host_get_prolongation(hg, d)):
                    assert np.array_equal(a, b), d
    finally:
        L.lbmg_host_destroy(hc)
        L.lbmg_host_destroy(hg)


@pytest.mark.parametrize("mesh", ["knot", "sheets"])
def test_gpu_pieces_assemble_the_same_matrices(mesh):
    V, F, depth = MESHES[mesh]()
    t = 1e-3
    hs = [L.lbmg_build_hierarchy(V, F, depth, gpu_clip=g) for g in (0, 1)]
    try:
        for h in hs:
            L.lbmg_assemble(h, t)
        d0, D = L.lbmg_levels(hs[0])
        for d in (D, D - 1, d0):
            mats = []
            for h in hs:
                rp, ci, M, Lm = L.lbmg_get_matrix(h, d)
                n = len(rp) - 1
                mats.append((sp.csr_matrix((M, ci, rp), shape=(n, n)), sp.csr_matrix((Lm, ci, rp), shape=(n, n))))
            for a, b in zip(mats[0], mats[1]):
                assert abs(a - b).max() <= 1e-13 * abs(a).max(), d
    finally:
        for h in hs:
            L.lbmg_destroy(h)
