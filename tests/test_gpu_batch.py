"""Batched solve against the FP64 oracle, mesh by mesh.

Many meshes of uneven size and depth share one hierarchy, aligned at the finest level:
batch level B - k holds level depth_i - k of every mesh i that has one.  Every member is
compared with its own oracle hierarchy (Sections 3.2 and 4 built by the oracle from
the member's mesh alone):
- the functions of its rows on every level are the oracle's functions;
- its M and L on every level equal the oracle's quadrature (1e-12 of the largest entry),
  and no entry couples two meshes;
- its prolongation on every level is the oracle's (Eq. 4);
- its right-hand side is the oracle's projection;
- its block of the batch solution (mixed precision, 1e-6 per mesh, V-cycles in one
  persistent launch or CG) matches the direct solution of the oracle's system in the
  M-norm to 1e-5.
Besides five small meshes, the batch holds two depth-7 members of the seeded 64-mesh
workload (a knot and a torus, 10k-11k triangles), so the persistent kernel's wide levels
run.  Vertex evaluation is compared with single-mesh handles.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import oracle
import paper_1505_03615_gb300 as L
from tests._match import permutation

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
T = 1e-2


def _meshes():
    mix = meshgen.batch_mix(64)
    return [
        (*meshgen.icosphere(2, 1.0, 1e-3, 1), 4),
        (*meshgen.torus_knot_tube(2, 3, 1.0, 0.12, 48, 8, 1e-6, 3), 5),
        (*meshgen.torus(1.0, 0.3, 60, 20, 1e-6, 5), 5),
        (*meshgen.ellipsoid((1.0, 0.6, 0.4), 2, 1e-6, 3), 3),
        (*meshgen.double_sheet(8, 0.05, 5, 0.5, 1e-6, 4), 5),
        mix[11],   # knot, 10,080 triangles, depth 7
        mix[27],   # torus, 11,234 triangles, depth 7
    ]


class Member:
    def __init__(self, hb, i, V, F, depth):
        self.V, self.F, self.depth = V, F, depth
        D, d0, nf, ro, vo = L.lbmg_instance_info(hb, i)
        assert D == depth
        self.d0, self.nfine, self.row_off, self.vert_off = d0, nf, ro, vo
        self.o = oracle.Hierarchy(V, F, depth, min_depth=d0)
        assert (self.o.min_depth, self.o.depth) == (d0, depth)


@pytest.fixture(scope="module")
def batch():
    meshes = _meshes()
    hb = L.lbmg_build_batch(meshes)
    L.lbmg_assemble(hb, T)
    members = [Member(hb, i, V, F, d) for i, (V, F, d) in enumerate(meshes)]
    yield meshes, hb, members
    L.lbmg_destroy(hb)


def _levels(hb, members):
    """(batch level, member, the member's own level, its rows at that batch level, perm to oracle)"""
    B0, BD = L.lbmg_levels(hb)
    for dB in range(B0, BD + 1):
        inst = L.lbmg_row_instances(hb, dB)
        corner, mintri = L.lbmg_get_dofs(hb, dB)
        for i, m in enumerate(members):
            real = m.depth - (BD - dB)
            rows = np.flatnonzero(inst == i)
            if real < m.d0:
                assert rows.size == 0
                continue
            oc, om = m.o.dofs(real)
            perm = permutation(corner[rows], mintri[rows], oc, om, m.F.shape[0])
            yield dB, i, m, real, rows, perm


def test_every_member_has_the_oracles_functions_on_every_level(batch):
    meshes, hb, members = batch
    seen = 0
    for dB, i, m, real, rows, perm in _levels(hb, members):
        assert rows.size == m.o.ndof(real)
        assert (perm >= 0).all() and np.unique(perm).size == perm.size
        seen += 1
    assert seen == sum(m.depth - m.d0 + 1 for m in members)


def test_every_member_matrices_match_oracle_on_every_level(batch):
    """Entry by entry at 1e-12 of the largest entry; rows of one mesh never reach another."""
    meshes, hb, members = batch
    B0, BD = L.lbmg_levels(hb)
    cache = {}
    for dB, i, m, real, rows, perm in _levels(hb, members):
        if dB not in cache:
            rp, ci, Mv, Lv = L.lbmg_get_matrix(hb, dB)
            n = rp.size - 1
            inst = L.lbmg_row_instances(hb, dB)
            r_of = np.repeat(np.arange(n), np.diff(rp))
            assert (inst[r_of] == inst[ci]).all()
            cache[dB] = (sp.csr_matrix((Mv, ci, rp), shape=(n, n)), sp.csr_matrix((Lv, ci, rp), shape=(n, n)))
        Mb, Lb = cache[dB]
        Mo, Lo = m.o.matrices(real)
        for got, ref in ((Mb[rows][:, rows], Mo[perm][:, perm]), (Lb[rows][:, rows], Lo[perm][:, perm])):
            assert abs(got - ref).max() <= 1e-12 * abs(ref).max()


def test_every_member_prolongation_matches_oracle(batch):
    meshes, hb, members = batch
    lev = {}
    for dB, i, m, real, rows, perm in _levels(hb, members):
        lev[(dB, i)] = (real, rows, perm)
    for (dB, i), (real, rows, perm) in lev.items():
        m = members[i]
        if real == m.d0:
            continue
        creal, crows, cperm = lev[(dB - 1, i)]
        assert creal == real - 1
        par, w = L.lbmg_get_prolongation(hb, dB)
        nc_b = L.lbmg_level_info(hb, dB - 1)[0]
        to_local = np.full(nc_b, -1)
        to_local[crows] = np.arange(crows.size)
        p, ww = par[rows], w[rows]
        r_idx, k_idx = np.nonzero(p >= 0)
        cols = to_local[p[r_idx, k_idx]]
        assert (cols >= 0).all()                       # parents are the mesh's own functions
        got = sp.csr_matrix((ww[r_idx, k_idx], (r_idx, cols)), shape=(rows.size, crows.size))
        P = m.o.prolongation(real)                      # oracle: (n_real, n_real-1)
        ref = P[perm][:, cperm]
        assert abs(got - ref).max() <= 1e-15


def _rhs(hb, meshes, nrhs_fn):
    f = np.concatenate([nrhs_fn(V) for V, F, d in meshes], axis=0)
    nu = sum(L.lbmg_instance_info(hb, i)[2] for i in range(len(meshes)))
    rhs = torch.zeros((nu, f.shape[1]), dtype=torch.float64, device=DEV)
    L.lbmg_project_rhs(hb, torch.tensor(f, device=DEV), rhs)
    return rhs


def _finest_perm(hb, m, i):
    """permutation of member i's user-ordered finest block to the oracle's finest order"""
    _, BD = L.lbmg_levels(hb)
    inst = L.lbmg_row_instances(hb, BD)
    corner, mintri = L.lbmg_get_dofs(hb, BD)
    rows = np.flatnonzero(inst == i)
    oc, om = m.o.dofs(m.depth)
    return permutation(corner[rows], mintri[rows], oc, om, m.F.shape[0])


def test_every_member_rhs_matches_oracle(batch):
    meshes, hb, members = batch
    rhs = _rhs(hb, meshes, lambda V: V).cpu().numpy()
    for i, m in enumerate(members):
        perm = _finest_perm(hb, m, i)
        ref = m.o.project_rhs(m.V)[perm]
        got = rhs[m.row_off:m.row_off + m.nfine]
        assert np.abs(got - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("solver", ["vcycle", "pcg"])
def test_every_member_solution_matches_oracle_direct_solve(batch, solver):
    """Mixed precision to 1e-6 per mesh and right-hand side; each member's block against the
    direct solution of the oracle's (M + t L) x = int f b in the M-norm, 1e-5."""
    meshes, hb, members = batch
    rhs = _rhs(hb, meshes, lambda V: V)
    x = torch.zeros_like(rhs)
    solve = L.lbmg_solve_pcg if solver == "pcg" else L.lbmg_solve
    code, st = solve(hb, rhs, x, 1e-6, 3000, L.LBMG_MIXED)
    assert code == L.LBMG_OK and st.converged
    rel = L.lbmg_instance_residuals(hb, 3)
    assert rel.shape == (len(meshes), 3) and np.all(rel <= 1e-6)
    xh = x.cpu().numpy()
    for i, m in enumerate(members):
        perm = _finest_perm(hb, m, i)
        Mo, Lo = m.o.matrices(m.depth)
        ref = spla.splu((Mo + T * Lo).tocsc()).solve(m.o.project_rhs(m.V))
        xo = np.zeros_like(ref)
        xo[perm] = xh[m.row_off:m.row_off + m.nfine]
        e = xo - ref
        err = np.sqrt(np.einsum("ij,ij->", e, Mo @ e) / np.einsum("ij,ij->", ref, Mo @ ref))
        assert err < 1e-5, (i, err)


def test_batch_vertex_evaluation_matches_single_meshes(batch):
    meshes, hb, members = batch
    nu = sum(m.nfine for m in members)
    nv = sum(V.shape[0] for V, _, _ in meshes)
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(size=(nu, 2)), device=DEV)
    u = torch.zeros((nv, 2), dtype=torch.float64, device=DEV)
    L.lbmg_eval_vertices(hb, x, u)
    for i, (V, F, d) in enumerate(meshes):
        m = members[i]
        h = L.lbmg_build_hierarchy(V, F, d)
        try:
            assert L.lbmg_level_info(h, d)[0] == m.nfine
            u1 = torch.zeros((V.shape[0], 2), dtype=torch.float64, device=DEV)
            L.lbmg_eval_vertices(h, x[m.row_off:m.row_off + m.nfine].contiguous(), u1)
            assert torch.allclose(u[m.vert_off:m.vert_off + V.shape[0]], u1, rtol=0, atol=1e-14)
        finally:
            L.lbmg_destroy(h)


def test_batch_pcg_takes_no_more_iterations_than_vcycles(batch):
    meshes, hb, members = batch
    rhs = _rhs(hb, meshes, lambda V: V)
    x = torch.zeros_like(rhs)
    code, st = L.lbmg_solve_pcg(hb, rhs, x, 1e-6, 1000, L.LBMG_MIXED)
    xv = torch.zeros_like(rhs)
    code_v, st_v = L.lbmg_solve(hb, rhs, xv, 1e-6, 3000, L.LBMG_MIXED)
    assert code == code_v == L.LBMG_OK and st.cycles <= st_v.cycles
