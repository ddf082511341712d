"""The mixed solve's outer residual with FP64 values carried as pairs of FP32 numbers
(lbmg_residual_split), against the FP64 residual of the same level (lbmg_residual, itself
pinned to the oracle's matrices in tests/test_gpu_parity.py).

Error bound: each product is a x = ah xh + (ah xl + al xh + exact error of ah xh) with the
al xl term dropped (|al xl| <= 2^-48 |a x|) and the small terms rounded in FP32, and every
sum is a two-sum pair, so the computed sum differs from the exact one by a few 2^-44 of
sum_j |a_ij x_j|; b - sum is then formed in FP64.  The test allows 2^-40 of
|b_i| + sum_j |a_ij x_j|, at a random iterate and at the solution (where the residual is all
cancellation)."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.mark.parametrize("nrhs", [1, 2, 3])
def test_split_residual_matches_fp64_residual(nrhs):
    V, F = meshgen.torus_knot_tube(2, 3, 1.0, 0.08, 200, 24, 1e-6, 2)
    h = L.lbmg_build_hierarchy(V, F, 6, min_depth=2)
    try:
        t = 1e-3
        L.lbmg_assemble(h, t)
        d0, D = L.lbmg_levels(h)
        rng = np.random.default_rng(nrhs)
        for d in range(d0 + 1, D + 1):
            rp, ci, Mv, Lv = L.lbmg_get_matrix(h, d)
            n = len(rp) - 1
            A = sp.csr_matrix((Mv + t * Lv, ci, rp), shape=(n, n))
            b = rng.normal(size=(n, nrhs))
            for x in (rng.normal(size=(n, nrhs)) * 1e3, spla.splu((A + 1e-12 * sp.identity(n)).tocsc()).solve(b)):
                bd, xd = torch.tensor(b, device=DEV), torch.tensor(np.ascontiguousarray(x), device=DEV)
                r64, rsp = torch.zeros_like(bd), torch.zeros_like(bd)
                L.lbmg_residual(h, d, bd, xd, r64)
                L.lbmg_residual_split(h, d, bd, xd, rsp)
                scale = np.abs(b) + abs(A) @ np.abs(x)
                err = np.abs(rsp.cpu().numpy() - r64.cpu().numpy())
                assert (err <= 2.0 ** -40 * scale).all(), (d, float((err / scale).max()))
        # the coarsest level has no packed copy
        n0 = L.lbmg_level_info(h, d0)[0]
        z = torch.zeros((n0, nrhs), dtype=torch.float64, device=DEV)
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_residual_split(h, d0, z, z, z.clone())
        assert e.value.code == 1
    finally:
        L.lbmg_destroy(h)
