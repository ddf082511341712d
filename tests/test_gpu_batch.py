"""Batched solve: many meshes of uneven size in one hierarchy and one persistent
launch give, mesh by mesh, the same functions, matrices and solutions as
separate single-mesh hierarchies (and hence as the oracle, which those match)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


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
    t = 1e-2
    hb = L.lbmg_build_batch(meshes)
    L.lbmg_assemble(hb, t)
    singles = []
    for V, F, d in meshes:
        h = L.lbmg_build_hierarchy(V, F, d)
        L.lbmg_assemble(h, t)
        singles.append(h)
    yield meshes, t, hb, singles
    L.lbmg_destroy(hb)
    for h in singles:
        L.lbmg_destroy(h)


def test_batch_layout(batch):
    meshes, t, hb, singles = batch
    assert L.lbmg_instances(hb) == len(meshes)
    off = 0
    voff = 0
    for i, (V, F, d) in enumerate(meshes):
        D, d0, nf, ro, vo = L.lbmg_instance_info(hb, i)
        n1 = L.lbmg_level_info(singles[i], d)[0]
        assert (D, nf, ro, vo) == (d, n1, off, voff)
        assert d0 == L.lbmg_levels(singles[i])[0]
        off += nf
        voff += V.shape[0]


def _stack(meshes, fn):
    return np.concatenate([fn(V) for V, F, d in meshes], axis=0)


def test_batch_rhs_and_solution_match_single_meshes(batch):
    """Mixed-precision batch solve to 1e-6 per mesh (the batched workload's target); each
    mesh's block of the solution matches that mesh's own direct solution in the M-norm."""
    meshes, t, hb, singles = batch
    f = _stack(meshes, lambda V: V)                      # x, y, z per vertex, meshes concatenated
    nu = sum(L.lbmg_level_info(h, d)[0] for h, (_, _, d) in zip(singles, meshes))
    rhs = torch.zeros((nu, 3), dtype=torch.float64, device=DEV)
    L.lbmg_project_rhs(hb, torch.tensor(f, device=DEV), rhs)
    x = torch.zeros_like(rhs)
    code, st = L.lbmg_solve(hb, rhs, x, 1e-6, 3000, L.LBMG_MIXED)
    assert code == L.LBMG_OK and st.converged
    rel = L.lbmg_instance_residuals(hb, 3)
    assert rel.shape == (len(meshes), 3) and np.all(rel <= 1e-6)
    off = 0
    for i, (V, F, d) in enumerate(meshes):
        n1 = L.lbmg_level_info(singles[i], d)[0]
        r1 = torch.zeros((n1, 3), dtype=torch.float64, device=DEV)
        L.lbmg_project_rhs(singles[i], torch.tensor(V, device=DEV), r1)
        assert torch.allclose(rhs[off:off + n1], r1, rtol=0, atol=1e-14 * r1.abs().max().item())
        rp, ci, M, Lm = L.lbmg_get_matrix(singles[i], d)
        Mm = sp.csr_matrix((M, ci, rp), shape=(n1, n1))
        A = (Mm + t * sp.csr_matrix((Lm, ci, rp), shape=(n1, n1))).tocsc()
        ref = spla.splu(A).solve(r1.cpu().numpy())
        e = x[off:off + n1].cpu().numpy() - ref
        err = np.sqrt(np.einsum("ij,ij->", e, Mm @ e) / np.einsum("ij,ij->", ref, Mm @ ref))
        assert err < 1e-5
        off += n1


def test_batch_vertex_evaluation(batch):
    meshes, t, hb, singles = batch
    nu = sum(L.lbmg_level_info(h, d)[0] for h, (_, _, d) in zip(singles, meshes))
    nv = sum(V.shape[0] for V, _, _ in meshes)
    rng = np.random.default_rng(0)
    x = torch.tensor(rng.normal(size=(nu, 2)), device=DEV)
    u = torch.zeros((nv, 2), dtype=torch.float64, device=DEV)
    L.lbmg_eval_vertices(hb, x, u)
    off = voff = 0
    for i, (V, F, d) in enumerate(meshes):
        n1 = L.lbmg_level_info(singles[i], d)[0]
        u1 = torch.zeros((V.shape[0], 2), dtype=torch.float64, device=DEV)
        L.lbmg_eval_vertices(singles[i], x[off:off + n1].contiguous(), u1)
        assert torch.allclose(u[voff:voff + V.shape[0]], u1, rtol=0, atol=1e-14)
        off += n1
        voff += V.shape[0]


def test_batch_pcg_matches_single_meshes(batch):
    """Conjugate gradients on the batch, each mesh with its own step lengths, preconditioned
    by the batched V-cycle: every mesh reaches 1e-6 and its block matches its own direct
    solution (M-norm 1e-5), in no more iterations than the batched V-cycle solve."""
    meshes, t, hb, singles = batch
    f = _stack(meshes, lambda V: V)
    nu = sum(L.lbmg_level_info(h, d)[0] for h, (_, _, d) in zip(singles, meshes))
    rhs = torch.zeros((nu, 3), dtype=torch.float64, device=DEV)
    L.lbmg_project_rhs(hb, torch.tensor(f, device=DEV), rhs)
    x = torch.zeros_like(rhs)
    code, st = L.lbmg_solve_pcg(hb, rhs, x, 1e-6, 1000, L.LBMG_MIXED)
    assert code == L.LBMG_OK and st.converged
    rel = L.lbmg_instance_residuals(hb, 3)
    assert np.all(rel <= 1e-6)
    xv = torch.zeros_like(rhs)
    code_v, st_v = L.lbmg_solve(hb, rhs, xv, 1e-6, 3000, L.LBMG_MIXED)
    assert code_v == L.LBMG_OK and st.cycles <= st_v.cycles
    off = 0
    for i, (V, F, d) in enumerate(meshes):
        n1 = L.lbmg_level_info(singles[i], d)[0]
        rp, ci, M, Lm = L.lbmg_get_matrix(singles[i], d)
        Mm = sp.csr_matrix((M, ci, rp), shape=(n1, n1))
        A = (Mm + t * sp.csr_matrix((Lm, ci, rp), shape=(n1, n1))).tocsc()
        ref = spla.splu(A).solve(rhs[off:off + n1].cpu().numpy())
        e = x[off:off + n1].cpu().numpy() - ref
        assert np.sqrt(np.einsum("ij,ij->", e, Mm @ e) / np.einsum("ij,ij->", ref, Mm @ ref)) < 1e-5
        off += n1
