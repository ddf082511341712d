"""Parity of the library's host hierarchy build with the FP64 oracle, on the CPU.

The host-only handle runs the same construction as the device handle: voxel pieces,
split functions per connected component (Section 4.2), the prolongation of Eq. 4 and
every level's sparsity pattern. Here it is compared with the oracle without a GPU:
- the same functions on every level;
- the same stored pattern;
- the same prolongation, entry for entry.
The rows are also checked to be in the order the coloured Gauss-Seidel sweep needs.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import oracle
import paper_1505_03615_gb300 as L
from tests._match import permutation

CASES = {
    "sphere": (lambda: meshgen.icosphere(3, 1.0, 1e-3, 1), 5, 2, True),
    "knot": (lambda: meshgen.torus_knot_tube(2, 3, 1.0, 0.12, 48, 8, 1e-6, 3), 5, 1, True),
    "sheets": (lambda: meshgen.double_sheet(20, 0.05, 6, 0.5, 1e-6, 4), 6, 2, True),
    "sheets_unsplit": (lambda: meshgen.double_sheet(20, 0.05, 6, 0.5, 1e-6, 4), 6, 2, False),
}


class HostCase:
    def __init__(self, name):
        build, depth, min_depth, split = CASES[name]
        self.V, self.F = build()
        self.h = L.lbmg_host_build(self.V, self.F, depth, min_depth=min_depth, split=int(split))
        self.o = oracle.Hierarchy(self.V, self.F, depth, min_depth=min_depth, split=split)
        self.d0, self.D = L.lbmg_host_levels(self.h)
        self.perm = {}
        for d in range(self.d0, self.D + 1):
            c, m = L.lbmg_host_get_dofs(self.h, d)
            oc, om = self.o.dofs(d)
            self.perm[d] = permutation(c, m, oc, om, self.F.shape[0])

    def n(self, d):
        return L.lbmg_host_level_info(self.h, d)[0]


@pytest.fixture(scope="module", params=sorted(CASES))
def case(request):
    c = HostCase(request.param)
    yield c
    L.lbmg_host_destroy(c.h)


def test_same_levels_and_split_functions(case):
    assert (case.d0, case.D) == (case.o.min_depth, case.o.depth)
    for d in range(case.d0, case.D + 1):
        assert case.n(d) == case.o.ndof(d)
        p = case.perm[d]
        assert (p >= 0).all() and len(np.unique(p)) == case.n(d)


def test_same_sparsity_pattern_on_every_level(case):
    for d in range(case.d0, case.D + 1):
        rp, ci = L.lbmg_host_get_pattern(case.h, d)
        n = case.n(d)
        assert rp[0] == 0 and rp[-1] == ci.size == L.lbmg_host_level_info(case.h, d)[1]
        # columns sorted and distinct within each row
        for i in range(0, n, max(1, n // 200)):
            row = ci[rp[i]:rp[i + 1]]
            assert (np.diff(row) > 0).all()
        p = case.perm[d]
        rows = np.repeat(np.arange(n), np.diff(rp))
        lib = sp.csr_matrix((np.ones(ci.size), (p[rows], p[ci])), shape=(n, n))
        Mo, _ = case.o.matrices(d)
        orc = sp.csr_matrix((np.ones(Mo.nnz), Mo.indices, Mo.indptr), shape=(n, n))
        assert lib.nnz == orc.nnz
        assert abs(lib - orc).max() == 0


def test_same_prolongation(case):
    for d in range(case.d0 + 1, case.D + 1):
        par, w = L.lbmg_host_get_prolongation(case.h, d)
        n = case.n(d)
        rows = np.repeat(np.arange(n), 8)
        m = par.ravel() >= 0
        P = sp.csr_matrix((w.ravel()[m], (rows[m], par.ravel()[m])), shape=(n, case.n(d - 1)))
        Po = case.o.prolongation(d)[case.perm[d]][:, case.perm[d - 1]]
        assert abs(P - Po).max() == 0


def test_rows_sorted_by_colour_and_one_colour_never_couples(case):
    """Rows come in corner-parity colour order, and the pattern has no entry between two
    different rows of one colour, so each colour is one exact parallel Gauss-Seidel step."""
    for d in range(case.d0 + 1, case.D + 1):
        corner, _ = L.lbmg_host_get_dofs(case.h, d)
        colour = (corner[:, 0] & 1) | ((corner[:, 1] & 1) << 1) | ((corner[:, 2] & 1) << 2)
        assert (np.diff(colour) >= 0).all()
        rp, ci = L.lbmg_host_get_pattern(case.h, d)
        rows = np.repeat(np.arange(case.n(d)), np.diff(rp))
        same = colour[rows] == colour[ci]
        assert (rows[same] == ci[same]).all()


def test_host_handle_rejects_bad_levels_and_inputs():
    V, F = meshgen.icosphere(2)
    h = L.lbmg_host_build(V, F, 4)
    try:
        d0, D = L.lbmg_host_levels(h)
        for d in (d0 - 1, D + 1):
            with pytest.raises(L.LbmgError):
                L.lbmg_host_level_info(h, d)
        with pytest.raises(L.LbmgError):
            L.lbmg_host_get_prolongation(h, d0)
    finally:
        L.lbmg_host_destroy(h)
    bad = F.copy()
    bad[0, 0] = V.shape[0]
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_host_build(V, bad, 4)
    assert e.value.code == 1
