"""Launch shapes, the launch-shape autotuner, and chained (programmatic dependent)
launches of the V-cycle.

Every launch shape computes the same Gauss-Seidel update and residual; only the
order of the additions inside a row changes.  So an FP64 sweep agrees with the
numpy colour-by-colour sweep to 1e-11 relative for every shape (as in the parity
tests), an FP32 sweep to 1e-4, and an FP64 residual with b - A x to 1e-12 of
the largest entry.  Programmatic dependent launch changes when a kernel starts,
not what it computes: solves with and without it are bitwise identical."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _knot():
    return meshgen.torus_knot_tube(2, 3, 1.0, 0.12, 48, 8, 1e-6, 3)


def _dev(a):
    return torch.tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _rel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _system(h, d, t):
    rp, ci, M, Lm = L.lbmg_get_matrix(h, d)
    n = len(rp) - 1
    Mm = sp.csr_matrix((M, ci, rp), shape=(n, n))
    return Mm, (Mm + t * sp.csr_matrix((Lm, ci, rp), shape=(n, n))).tocsr()


def _colour_sweeps(A, corner, b, x, sweeps, floor=1e-20):
    """Colour-by-colour Gauss-Seidel; rows whose diagonal is not positive or below
    floor * mean diagonal are not relaxed (the library's rule for sliver functions)."""
    x = x.copy()
    colour = (corner[:, 0] & 1) | ((corner[:, 1] & 1) << 1) | ((corner[:, 2] & 1) << 2)
    dg = A.diagonal()
    keep = (dg > 0) & (dg >= floor * dg.mean())
    dinv = np.where(keep, 1.0 / np.where(keep, dg, 1.0), 0.0)
    for _ in range(sweeps):
        for c in range(8):
            rows = np.where(colour == c)[0]
            x[rows] += dinv[rows, None] * (b[rows] - A[rows] @ x)
    return x


@pytest.fixture(scope="module")
def knot():
    V, F = _knot()
    h = L.lbmg_build_hierarchy(V, F, 5, min_depth=1)
    L.lbmg_assemble(h, 1e-2)
    yield V, F, h
    L.lbmg_destroy(h)


@pytest.mark.parametrize("tpr", [4, 8, 16])
@pytest.mark.parametrize("tpb", [128, 256, 512])
def test_every_launch_shape_matches_reference_sweep_and_residual(knot, tpr, tpb):
    V, F, h = knot
    d0, D = L.lbmg_levels(h)
    try:
        for d in (D, d0 + 1):
            for prec in (L.LBMG_FP64, L.LBMG_MIXED):
                for kind in (0, 1):
                    L.lbmg_set_launch_shape(h, d, prec, kind, tpr, tpb)
            assert L.lbmg_launch_shape(h, d, L.LBMG_FP64) == ((tpr, tpb), (tpr, tpb))
            _, A = _system(h, d, 1e-2)
            n = A.shape[0]
            corner, _ = L.lbmg_get_dofs(h, d)
            rng = np.random.default_rng(3)
            b = A @ rng.normal(size=(n, 3))
            x0 = np.zeros((n, 3))
            xr = _colour_sweeps(A, corner, b, x0, 2)
            x = _dev(x0)
            L.lbmg_smooth(h, d, _dev(b), x, 2, L.LBMG_FP64)
            assert _rel(x.cpu().numpy(), xr) <= 1e-11
            x32 = _dev(x0)
            L.lbmg_smooth(h, d, _dev(b), x32, 2, L.LBMG_MIXED)
            assert _rel(x32.cpu().numpy(), xr) <= 1e-4
            xs = rng.normal(size=(n, 3))
            r = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
            L.lbmg_residual(h, d, _dev(b), _dev(xs), r)
            assert np.abs(r.cpu().numpy() - (b - A @ xs)).max() <= 1e-12 * np.abs(b).max()
    finally:
        for d in range(d0 + 1, D + 1):
            for prec in (L.LBMG_FP64, L.LBMG_MIXED):
                for kind in (0, 1):
                    L.lbmg_set_launch_shape(h, d, prec, kind, 4, 256)


def test_invalid_launch_shapes_are_rejected(knot):
    _, _, h = knot
    _, D = L.lbmg_levels(h)
    for tpr, tpb in ((5, 256), (8, 100), (8, 1024), (32, 256)):
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_set_launch_shape(h, D, L.LBMG_MIXED, 0, tpr, tpb)
        assert e.value.code == 1


@pytest.mark.parametrize("graphs", [1, 0])
def test_dependent_launch_changes_no_bit(graphs):
    """On a side stream (the legacy default stream takes no programmatic serialization,
    so direct launches there fall back to plain stream order)."""
    V, F = _knot()
    hs = [L.lbmg_build_hierarchy(V, F, 5, min_depth=1, pdl=p, use_graphs=graphs) for p in (1, 0)]
    side = torch.cuda.Stream()
    try:
        with torch.cuda.stream(side):
            _compare_solves(V, hs)
    finally:
        for h in hs:
            L.lbmg_destroy(h)


def _compare_solves(V, hs):
    n = None
    for h in hs:
        L.lbmg_assemble(h, 1e-2)
        n = L.lbmg_level_info(h, 5)[0]
    rhs = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    L.lbmg_project_rhs(hs[0], _dev(V), rhs)
    for prec in (L.LBMG_MIXED, L.LBMG_FP64):
        xs = []
        for h in hs:
            x = torch.zeros_like(rhs)
            L.lbmg_vcycles(h, rhs, x, 7, prec)
            xs.append(x)
        assert torch.equal(xs[0], xs[1])
    res = []
    for h in hs:
        x = torch.zeros_like(rhs)
        code, st = L.lbmg_solve(h, rhs, x, 1e-6, 3000, L.LBMG_MIXED)
        assert code == L.LBMG_OK
        res.append((x, st.cycles))
    assert res[0][1] == res[1][1] and torch.equal(res[0][0], res[1][0])


def test_autotuned_shapes_are_valid_cached_and_solve_correctly(tmp_path):
    V, F = meshgen.torus_knot_tube(2, 3, 1.0, 0.06, 200, 20, 1e-6, 3)
    depth, t = 7, 1e-3
    h1 = L.lbmg_build_hierarchy(V, F, depth)
    h2 = L.lbmg_build_hierarchy(V, F, depth)
    try:
        for h in (h1, h2):
            L.lbmg_assemble(h, t)
        d0, D = L.lbmg_levels(h1)
        timed = L.lbmg_autotune(h1, 3, L.LBMG_MIXED, reps=2)
        assert timed == 2 * (D - d0)
        shapes = [L.lbmg_launch_shape(h1, d, L.LBMG_MIXED) for d in range(d0 + 1, D + 1)]
        for s in shapes:
            for tpr, tpb in s:
                assert tpr in (4, 8, 16) and tpb in (128, 256, 512)
        # identical levels of another handle come from the cache
        assert L.lbmg_autotune(h2, 3, L.LBMG_MIXED, reps=2) == 0
        assert [L.lbmg_launch_shape(h2, d, L.LBMG_MIXED) for d in range(d0 + 1, D + 1)] == shapes
        path = tmp_path / "tune.txt"
        L.lbmg_tune_cache_save(str(path))
        assert len([ln for ln in path.read_text().splitlines() if not ln.startswith("#")]) >= 2 * (D - d0)
        L.lbmg_tune_cache_load(str(path))
        # the tuned solve still reaches the direct solution
        n = L.lbmg_level_info(h1, D)[0]
        rhs = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
        L.lbmg_project_rhs(h1, _dev(V), rhs)
        x = torch.zeros_like(rhs)
        code, st = L.lbmg_solve(h1, rhs, x, 1e-6, 3000, L.LBMG_MIXED)
        assert code == L.LBMG_OK and st.converged
        Mm, A = _system(h1, D, t)
        xd = spla.splu(A.tocsc()).solve(rhs.cpu().numpy())
        e = x.cpu().numpy() - xd
        assert np.sqrt(np.einsum("ij,ij->", e, Mm @ e) / np.einsum("ij,ij->", xd, Mm @ xd)) <= 1e-5
    finally:
        L.lbmg_destroy(h1)
        L.lbmg_destroy(h2)


@pytest.mark.parametrize("graphs", [1, 0])
def test_whole_sweep_kernel_changes_no_bit(graphs):
    """The whole-sweep cooperative kernel (shape 4 x 1024: every colour step of a smoothing in
    one launch, blocks meeting at a bounded grid barrier) computes exactly what the colour
    launches of 4 threads per row compute; it is refused for FP64 sweeps and for residuals."""
    V, F = _knot()
    h = L.lbmg_build_hierarchy(V, F, 5, min_depth=1, use_graphs=graphs)
    try:
        L.lbmg_assemble(h, 1e-2)
        d0, D = L.lbmg_levels(h)
        n = L.lbmg_level_info(h, D)[0]
        rhs = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
        L.lbmg_project_rhs(h, _dev(V), rhs)
        xs = []
        for tpb in (256, 1024):
            for d in range(d0 + 1, D + 1):
                L.lbmg_set_launch_shape(h, d, L.LBMG_MIXED, 0, 4, tpb)
            x = torch.zeros_like(rhs)
            assert L.lbmg_vcycles(h, rhs, x, 5, L.LBMG_MIXED) == L.LBMG_OK
            code, st = L.lbmg_solve(h, rhs, torch.zeros_like(rhs), 1e-6, 3000, L.LBMG_MIXED)
            assert code == L.LBMG_OK
            xs.append((x, st.cycles))
        assert torch.equal(xs[0][0], xs[1][0]) and xs[0][1] == xs[1][1]
        for prec, kind in ((L.LBMG_FP64, 0), (L.LBMG_MIXED, 1)):
            with pytest.raises(L.LbmgError) as e:
                L.lbmg_set_launch_shape(h, D, prec, kind, 4, 1024)
            assert e.value.code == 1
    finally:
        L.lbmg_destroy(h)
