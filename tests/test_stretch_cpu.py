"""Oracle parity through a stretch of a large mesh, on the CPU (host-only hierarchy).

The library's host build of the 200k-triangle (2,3) knot at depth 8 is compared with the oracle
built on 20,000 consecutive triangles of it, on the full mesh's grid: on functions whose support
and neighbours' supports no outside triangle can meet, both have the same functions (corner and
smallest triangle) and the same sparsity pattern, row by row.  The same selection serves the GPU
test of the 4M-triangle workload's matrices and right-hand sides (tests/test_gpu_fullsize.py)."""
import numpy as np

import meshgen
import oracle
import paper_1505_03615_gb300 as L
from tests._stretch import complete_sample, oracle_to_library, stretch


def test_stretch_functions_and_patterns_match_the_full_build():
    V, F, depth, t, f, tol, _ = meshgen.config_mesh("knot23_200k_d8")
    t0, ntri = 60_000, 20_000
    S, centre = oracle.embedding_of(V)
    Vp, Fp = stretch(V, F, t0, ntri)
    o = oracle.Hierarchy(Vp, Fp, depth, min_depth=depth, embedding=(S, centre))
    oc, om = o.dofs(depth)
    pick = complete_sample(V, F, t0, ntri, S, centre, depth, oc, om, 300)
    assert len(pick) >= 200
    h = L.lbmg_host_build(V, F, depth)
    try:
        lc, lm = L.lbmg_host_get_dofs(h, depth)
        rp, ci = L.lbmg_host_get_pattern(h, depth)
    finally:
        L.lbmg_host_destroy(h)
    to_lib = oracle_to_library(oc, om.astype(np.int64) + t0, lc, lm, F.shape[0])
    Mo, _ = o.matrices(depth)
    Mo = Mo.tocsr()
    for io in pick:
        il = to_lib[io]
        assert il >= 0, io                            # the same function in the full build
        cols_o = Mo.indices[Mo.indptr[io]:Mo.indptr[io + 1]]
        mapped = to_lib[cols_o]
        assert (mapped >= 0).all(), io                # its neighbours too
        cols_l = ci[rp[il]:rp[il + 1]]
        assert np.array_equal(np.sort(mapped), np.sort(cols_l)), io
