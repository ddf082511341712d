"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these re-types the oracle's formulas: each compares it with a closed
form, an independent exact integration, brute force, or a textbook routine.
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.csgraph as csg
import scipy.sparse.linalg as spla

import meshgen
import oracle
from tests import _exact

pytestmark = pytest.mark.filterwarnings("ignore::DeprecationWarning")


def corner_positions(h, d):
    """Physical position of each dof's grid corner at depth d (embedding reading A5)."""
    corner, _ = h.dofs(d)
    side = h.cube_side / 2 ** d
    return corner * side - h.cube_side / 2 + h.center[None, :]


def tri_geometry(V, F):
    P = V[F]
    cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
    A = 0.5 * np.linalg.norm(cr, axis=1)
    return P, A, cr / (2 * A[:, None])


@pytest.fixture(scope="module")
def sphere_h(icosphere):
    V, F = icosphere
    return oracle.Hierarchy(V, F, 5, min_depth=2)


# --------------------------------------------------------------------------
# assembly: closed forms (Eq. 2, Section 5.1)
# --------------------------------------------------------------------------

def test_mass_sums_to_area_on_every_level(icosphere, sphere_h):
    """1^T M 1 = surface area: the split hats form a partition of unity (Section 4.2)."""
    V, F = icosphere
    _, A, _ = tri_geometry(V, F)
    for d in sphere_h.levels():
        M, _ = sphere_h.matrices(d)
        assert abs(M.sum() - A.sum()) < 1e-12 * A.sum()


def test_stiffness_annihilates_constants(sphere_h):
    for d in sphere_h.levels():
        M, L = sphere_h.matrices(d)
        assert np.abs(L @ np.ones(L.shape[0])).max() < 1e-12 * np.abs(L.diagonal()).max()


def test_symmetric_positive_semidefinite(icosphere):
    V, F = icosphere
    h = oracle.Hierarchy(V, F, 3, min_depth=3)
    M, L = h.matrices(3)
    assert abs(M - M.T).max() == 0 or abs(M - M.T).max() < 1e-16
    assert abs(L - L.T).max() < 1e-14
    em = np.linalg.eigvalsh(M.toarray())
    el = np.linalg.eigvalsh(L.toarray())
    assert em.min() > 0
    assert el.min() > -1e-12 * el.max()


@pytest.mark.parametrize("a,b", [(0, 0), (1, 1), (2, 2), (0, 1), (0, 2), (1, 2)])
def test_stiffness_reproduces_tangential_metric(icosphere, sphere_h, a, b):
    """c_a^T L c_b = int <P e_a, P e_b> = sum_t A_t (delta_ab - n_a n_b): linear precision
    of the hats plus the tangential projection grad_M = (I - n n^T) grad."""
    V, F = icosphere
    _, A, n = tri_geometry(V, F)
    for d in sphere_h.levels():
        _, L = sphere_h.matrices(d)
        c = corner_positions(sphere_h, d)
        expect = (A * ((a == b) - n[:, a] * n[:, b])).sum()
        assert abs(c[:, a] @ L @ c[:, b] - expect) < 1e-11 * max(1.0, abs(expect))


@pytest.mark.parametrize("powers", [(2, 0, 0), (0, 0, 2), (2, 2, 0), (0, 2, 2), (2, 2, 2)])
def test_mass_reproduces_monomial_integrals(icosphere, sphere_h, powers):
    """c_f^T M c_f = int f^2 for f in {x, z, xy, yz, xyz}: trilinear precision of the hats
    with exact integration up to degree 6 (the rule must be exact for b_a b_b)."""
    V, F = icosphere
    P, A, _ = tri_geometry(V, F)
    half = tuple(p // 2 for p in powers)
    expect = sum(_exact.monomial_integral(P[t], powers) for t in range(F.shape[0]))
    for d in sphere_h.levels():
        M, _ = sphere_h.matrices(d)
        c = corner_positions(sphere_h, d)
        cf = np.prod([c[:, k] ** half[k] for k in range(3)], axis=0)
        assert abs(cf @ M @ cf - expect) < 1e-11 * abs(expect)


def _three_triangle_mesh():
    # an anchor triangle near the origin, a probe triangle strictly inside voxel
    # (2,2,2) of the depth-2 grid, and a far triangle that fixes the bounding box [0,1]^3
    V = np.array([[0, 0, 0], [0.2, 0, 0], [0, 0.2, 0],
                  [0.55, 0.56, 0.57], [0.70, 0.60, 0.58], [0.58, 0.72, 0.66],
                  [1, 1, 1], [0.9, 1, 1], [1, 0.9, 1]], dtype=np.float64)
    F = np.array([[0, 1, 2], [3, 4, 5], [6, 7, 8]], dtype=np.int32)
    return V, F


def test_single_voxel_entries_match_exact_integration():
    """Every M and L entry of a triangle inside one voxel equals the exact
    barycentric-monomial integral of the trilinear hats (Eq. 2, Section 5.1)."""
    V, F = _three_triangle_mesh()
    h = oracle.Hierarchy(V, F, 2, min_depth=2)
    M, L = h.matrices(2)
    tri, vox, _ = h.fragments(2)
    sel = np.where(tri == 1)[0]
    assert len(sel) == 1
    vx = vox[sel[0]]
    assert tuple(vx) == (2, 2, 2)
    key, ktri, kdof = h.corner_tri(2)
    N = 4
    dofs = []
    for a in range(8):
        c = vx + np.array([a & 1, (a >> 1) & 1, (a >> 2) & 1])
        k = (c[0] * (N + 1) + c[1]) * (N + 1) + c[2]
        dofs.append(int(kdof[(key == k) & (ktri == 1)][0]))
    side = h.cube_side / N
    lo = vx * side - h.cube_side / 2 + h.center
    Me, Le = _exact.hat_matrices_single_voxel(V[F[1]], lo, side)
    Mo = M[np.ix_(dofs, dofs)].toarray()
    Lo = L[np.ix_(dofs, dofs)].toarray()
    assert np.abs(Mo - Me).max() < 1e-13 * np.abs(Me).max()
    assert np.abs(Lo - Le).max() < 1e-12 * np.abs(Le).max()


# --------------------------------------------------------------------------
# hierarchy: nesting, prolongation (Sections 4.1, 4.3)
# --------------------------------------------------------------------------

def test_observation_parent_component_unique(sphere_h):
    assert sphere_h.check_nesting() == 0


def test_galerkin_identity(sphere_h):
    """Nesting of the split spaces (Claim, Section 4.1) with Eq. 4's prolongation:
    M_{d-1} = P^T M_d P and L_{d-1} = P^T L_d P, both sides assembled directly."""
    for d in sphere_h.levels()[1:]:
        P = sphere_h.prolongation(d)
        Mf, Lf = sphere_h.matrices(d)
        Mc, Lc = sphere_h.matrices(d - 1)
        assert abs(P.T @ Mf @ P - Mc).max() < 1e-13 * abs(Mc).max()
        assert abs(P.T @ Lf @ P - Lc).max() < 1e-12 * abs(Lc).max()


def _basis_values_at(h, d, V, F, t, bary):
    """Values of every dof of level d at the point with barycentrics `bary` in triangle t,
    evaluated from the definition b_k^i(p) = b_k(p) if p in C_k^i (Section 4.2)."""
    p = bary @ V[F[t]]
    N = 2 ** d
    side = h.cube_side / N
    g = (p - h.center + h.cube_side / 2) / side        # grid coordinates at depth d
    key, ktri, kdof = h.corner_tri(d)
    out = {}
    base = np.floor(g).astype(int)
    for a in range(8):
        c = base + np.array([a & 1, (a >> 1) & 1, (a >> 2) & 1])
        val = np.prod(np.maximum(0.0, 1.0 - np.abs(g - c)))
        if val <= 0:
            continue
        k = (c[0] * (N + 1) + c[1]) * (N + 1) + c[2]
        m = (key == k) & (ktri == t)
        assert m.sum() == 1
        out[int(kdof[m][0])] = val
    return out


def test_prolongation_refines_split_hats_pointwise(icosphere, sphere_h):
    """b_k^i(p) = sum_{k',i'} chi P(k,k') b_{k'}^{i'}(p) at random surface points (Eq. 4):
    this fixes the 1D stencil 1/2(1 2 1) of the trilinear hat and the parent choice."""
    V, F = icosphere
    rng = np.random.default_rng(0)
    for d in sphere_h.levels()[1:]:
        P = sphere_h.prolongation(d).tocsc()
        for _ in range(40):
            t = int(rng.integers(F.shape[0]))
            w = rng.dirichlet([1, 1, 1])
            fine = _basis_values_at(sphere_h, d, V, F, t, w)
            coarse = _basis_values_at(sphere_h, d - 1, V, F, t, w)
            # sum of all coarse values = 1 (partition of unity)
            assert abs(sum(coarse.values()) - 1) < 1e-12
            assert abs(sum(fine.values()) - 1) < 1e-12
            for j in set(coarse) | set(P[list(fine)].nonzero()[1]):
                col = P[:, j]
                val = sum(col[i, 0] * v for i, v in fine.items())
                assert abs(val - coarse.get(j, 0.0)) < 1e-12


def test_prolongation_weights_are_half_powers(sphere_h):
    for d in sphere_h.levels()[1:]:
        P = sphere_h.prolongation(d)
        cnt = np.diff(P.indptr)
        assert set(np.unique(cnt)).issubset({1, 2, 4, 8})
        for i in range(P.shape[0]):
            vals = P.data[P.indptr[i]:P.indptr[i + 1]]
            assert np.allclose(vals, 1.0 / cnt[i], rtol=0, atol=0)


# --------------------------------------------------------------------------
# connectivity-aware split (Section 4.2)
# --------------------------------------------------------------------------

def _refined_samples(V, F, R):
    """Vertices of an R-fold uniform refinement of each triangle, with shared edges merged."""
    pts, owner = [], []
    index = {}
    edges = []
    for t, (a, b, c) in enumerate(F):
        local = {}
        for i in range(R + 1):
            for j in range(R + 1 - i):
                k = R - i - j
                # canonical key: barycentric weights on sorted vertex ids
                w = {a: i, b: j, c: k}
                key = tuple(sorted((v, n) for v, n in w.items() if n > 0))
                if key not in index:
                    index[key] = len(pts)
                    pts.append((i * V[a] + j * V[b] + k * V[c]) / R)
                    owner.append(t)
                local[(i, j)] = index[key]
        for i in range(R + 1):
            for j in range(R + 1 - i):
                if i + j < R:
                    edges.append((local[(i, j)], local[(i + 1, j)]))
                    edges.append((local[(i, j)], local[(i, j + 1)]))
                    edges.append((local[(i + 1, j)], local[(i, j + 1)]))
    return np.array(pts), np.array(edges)


def _tri_samples(F, R):
    """For each triangle, the index list of its refined sample points (same order as above)."""
    out = []
    index = {}
    n = 0
    for t, (a, b, c) in enumerate(F):
        ids = []
        for i in range(R + 1):
            for j in range(R + 1 - i):
                k = R - i - j
                w = {a: i, b: j, c: k}
                key = tuple(sorted((v, m) for v, m in w.items() if m > 0))
                if key not in index:
                    index[key] = n
                    n += 1
                ids.append(index[key])
        out.append(ids)
    return out


def _flood_labels(g, edges, c, half):
    """Connected components of the refined sample graph restricted to the open box
    (c - half, c + half)^3; returns (local index of each sample or -1, labels)."""
    inside = np.all((g > c - half) & (g < c + half), axis=1)
    ids = np.where(inside)[0]
    loc = -np.ones(len(g), dtype=np.int64)
    loc[ids] = np.arange(len(ids))
    e = edges[inside[edges[:, 0]] & inside[edges[:, 1]]]
    G = sp.coo_matrix((np.ones(len(e)), (loc[e[:, 0]], loc[e[:, 1]])), shape=(len(ids), len(ids)))
    _, lab = csg.connected_components(G, directed=False)
    return loc, lab


@pytest.mark.parametrize("mesh", ["knot", "sheets"])
def test_split_components_match_flood_fill(mesh):
    """Components of supp(b_k) /\\ M (Section 4.2) against flood fill over a finely
    refined copy of the mesh.  Flood fill inside the open support cube can only miss
    connections through necks thinner than its sample spacing, and flood fill inside a
    cube enlarged by a tenth of a voxel can only add connections, so the oracle's split
    must lie between the two: joined by the first => joined by the oracle => joined
    by the second."""
    if mesh == "knot":
        V, F = meshgen.torus_knot_tube(2, 3, 1.0, 0.12, 48, 8, 1e-6, 3)
        depth = 3
    else:
        V, F = meshgen.double_sheet(6, 0.05, 4, 0.5, 1e-6, 9)
        depth = 4
    R = 12
    h = oracle.Hierarchy(V, F, depth, min_depth=depth)
    pts, edges = _refined_samples(V, F, R)
    tsamp = _tri_samples(F, R)
    N = 2 ** depth
    side = h.cube_side / N
    g = (pts - h.center + h.cube_side / 2) / side
    key, ktri, kdof = h.corner_tri(depth)
    checked = split_seen = 0
    for k in np.unique(key):
        c = np.array([k // ((N + 1) ** 2), (k // (N + 1)) % (N + 1), k % (N + 1)])
        loc, lab = _flood_labels(g, edges, c, 1.0)
        loc2, lab2 = _flood_labels(g, edges, c, 1.1)
        m = key == k
        items = []
        for t, dof in zip(ktri[m], kdof[m]):
            s = [loc[i] for i in tsamp[t] if loc[i] >= 0]
            s2 = [loc2[i] for i in tsamp[t] if loc2[i] >= 0]
            if s:
                items.append((int(dof), int(lab[s[0]]), int(lab2[s2[0]])))
        for i in range(len(items)):
            for j in range(i + 1, len(items)):
                inner = items[i][1] == items[j][1]
                same = items[i][0] == items[j][0]
                outer = items[i][2] == items[j][2]
                assert (not inner) or same
                assert (not same) or outer
                checked += 1
                split_seen += not same
    assert checked > 100 and split_seen > 10


def test_two_sheets_decouple_and_unsplit_couples():
    """Two parallel sheets half a voxel apart (teaser, Section 4): the split space gives
    block-diagonal M and L; the unsplit space of Section 3.2 couples the sheets."""
    V, F = meshgen.double_sheet(8, 0.05, 4, 0.5, 1e-6, 4)
    nt = F.shape[0]
    for split in (True, False):
        h = oracle.Hierarchy(V, F, 4, min_depth=2, split=split)
        for d in h.levels():
            M, L = h.matrices(d)
            key, ktri, kdof = h.corner_tri(d)
            sheet = np.zeros(h.ndof(d), dtype=np.int64)
            np.maximum.at(sheet, kdof, np.where(ktri < nt // 2, 1, 2))
            lower = np.zeros(h.ndof(d), dtype=np.int64)
            np.bitwise_or.at(lower, kdof, np.where(ktri < nt // 2, 1, 2))
            Mc = M.tocoo()
            cross = (lower[Mc.row] != lower[Mc.col]) & (lower[Mc.row] != 3) & (lower[Mc.col] != 3)
            if split:
                assert set(np.unique(lower)).issubset({1, 2})
                assert not cross.any()
            else:
                assert (lower == 3).any()


def test_same_corner_components_and_same_parity_never_couple(sphere_h):
    """Functions of one corner have disjoint supports; corners of equal parity
    (k mod 2) have disjoint supports: both give zero entries (8-colouring)."""
    for d in sphere_h.levels():
        M, L = sphere_h.matrices(d)
        corner, _ = sphere_h.dofs(d)
        Mc = M.tocoo()
        off = Mc.row != Mc.col
        same_parity = np.all((corner[Mc.row] % 2) == (corner[Mc.col] % 2), axis=1)
        assert not (off & same_parity).any()


# --------------------------------------------------------------------------
# right-hand side and vertex evaluation
# --------------------------------------------------------------------------

def test_rhs_of_constants_and_coordinates(icosphere, sphere_h):
    """int f b_i for f = 1 and f = x equals M 1 and M c_x (linear precision)."""
    V, F = icosphere
    d = sphere_h.depth
    M, _ = sphere_h.matrices(d)
    c = corner_positions(sphere_h, d)
    f = np.concatenate([np.ones((V.shape[0], 1)), V], axis=1)
    rhs = sphere_h.project_rhs(f)
    expect = np.stack([M @ np.ones(M.shape[0])] + [M @ c[:, k] for k in range(3)], axis=1)
    assert np.abs(rhs - expect).max() < 1e-13 * np.abs(expect).max()


def test_eval_vertices_reproduces_coordinates(icosphere, sphere_h):
    V, F = icosphere
    c = corner_positions(sphere_h, sphere_h.depth)
    u = sphere_h.eval_vertices(c)
    assert np.abs(u - V).max() < 1e-12


# --------------------------------------------------------------------------
# spectrum (Section 5.1)
# --------------------------------------------------------------------------

def _p1_fem(V, F):
    """Textbook P1 (cotangent) stiffness and consistent mass on the triangle mesh."""
    n = V.shape[0]
    LI, LJ, LV, MI, MJ, MV = [], [], [], [], [], []
    for tri in F:
        P = V[tri]
        area = 0.5 * np.linalg.norm(np.cross(P[1] - P[0], P[2] - P[0]))
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            u, v = P[j] - P[i], P[k] - P[i]
            half_cot = 0.5 * (u @ v) / np.linalg.norm(np.cross(u, v))
            a, b = tri[j], tri[k]
            LI += [a, b, a, b]; LJ += [b, a, a, b]; LV += [-half_cot, -half_cot, half_cot, half_cot]
        for a in range(3):
            for b in range(3):
                MI.append(tri[a]); MJ.append(tri[b]); MV.append(area / 6 if a == b else area / 12)
    L = sp.coo_matrix((LV, (LI, LJ)), shape=(n, n)).tocsr()
    M = sp.coo_matrix((MV, (MI, MJ)), shape=(n, n)).tocsr()
    return L, M


def _golden_sphere_spectrum():
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "sphere_spectrum.txt")
    rows = [line.split() for line in open(path) if line.strip() and not line.startswith("#")]
    return [(int(l), float(lam), int(mult)) for l, lam, mult in rows]


def test_sphere_spectrum_multiplicities(icosphere):
    """L x = lambda M x on the unit sphere: 0 once, then clusters of 3, 5, 7 near
    l(l+1) = 2, 6, 12 (Section 5.1), and close to the cotangent operator's values."""
    V, F = icosphere
    h = oracle.Hierarchy(V, F, 4, min_depth=4)
    M, L = h.matrices(4)
    w = sla.eigh(L.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 15])
    start = 0
    for l, lam, mult in _golden_sphere_spectrum():
        block = w[start:start + mult]
        if lam == 0:
            assert np.all(np.abs(block) < 1e-4)   # dense eigh on an ill-conditioned M; L 1 = 0 is pinned exactly above
        else:
            assert np.all(np.abs(block - lam) < 0.02 * lam)
            if start + mult < len(w):
                assert w[start + mult] > 1.3 * lam       # the cluster is complete
        start += mult
    Lc, Mc = _p1_fem(V, F)
    wc = sla.eigh(Lc.toarray(), Mc.toarray(), eigvals_only=True, subset_by_index=[0, 15])
    assert np.all(np.abs(w[1:] - wc[1:]) < 0.02 * wc[1:])


def test_spectrum_rotation_invariant(icosphere):
    """Spectrum barely moves when the model is rotated before embedding (Section 5.1)."""
    V, F = icosphere
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    out = []
    for VV in (V, V @ Q.T):
        h = oracle.Hierarchy(VV, F, 4, min_depth=4)
        M, L = h.matrices(4)
        out.append(sla.eigh(L.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 15]))
    assert np.all(np.abs(out[0][1:] - out[1][1:]) < 0.01 * out[0][1:])


# --------------------------------------------------------------------------
# solver (Sections 4.3, 5.2)
# --------------------------------------------------------------------------

def _mnorm(M, e):
    return float(np.sqrt(e @ (M @ e)))


def test_vcycle_converges_to_direct_solution(icosphere):
    """Plain V-cycles (Gauss-Seidel smoothing, Section 5.2) reach the direct solution.

    The restricted hats are nearly dependent where the surface is close to an
    axis-aligned plane (Discussion, Section 5), so the asymptotic rate is slow;
    the solution is compared in the M-norm, i.e. as a function on the surface."""
    V, F = icosphere
    h = oracle.Hierarchy(V, F, 5, min_depth=2)
    t = 1e-3
    f = meshgen.sphere_harmonic_rhs(V)
    rhs = h.project_rhs(f)
    x, cycles, hist = h.solve(t, rhs, tol=1e-10, max_cycles=800)
    M, L = h.matrices(5)
    A = (M + t * L).tocsc()
    xd = spla.spsolve(A, rhs[:, 0])
    assert hist[-1, 0] <= 1e-10
    assert _mnorm(M, x[:, 0] - xd) < 1e-8 * _mnorm(M, xd)
    # the residual never grows from one cycle to the next
    assert np.all(np.diff(hist[:, 0]) <= 0)


def test_vcycle_fixed_point_independent_of_coarsest_level(icosphere):
    V, F = icosphere
    f = meshgen.sphere_harmonic_rhs(V)
    xs = []
    for d0 in (2, 4):
        h = oracle.Hierarchy(V, F, 5, min_depth=d0)
        rhs = h.project_rhs(f)
        x, c, hist = h.solve(1e-3, rhs, tol=1e-11, max_cycles=1000)
        assert hist[-1, 0] <= 1e-11
        xs.append(x[:, 0])
    M, _ = h.matrices(5)
    assert _mnorm(M, xs[0] - xs[1]) < 1e-8 * _mnorm(M, xs[0])


def _tri_areas(V, F):
    e1 = V[F[:, 1]] - V[F[:, 0]]
    e2 = V[F[:, 2]] - V[F[:, 0]]
    return 0.5 * np.linalg.norm(np.cross(e1, e2), axis=1)


@pytest.mark.parametrize("mesh", ["sphere", "sheets"])
def test_weighted_mass_partition_of_unity(mesh):
    """The split functions sum to one on the surface, so for any triangle weights w the
    entries of the weighted mass matrix sum to sum_T w_T |T|, on every level; one triangle
    alone gives its own area (Section 5.3's M_t on the build-time space)."""
    if mesh == "sphere":
        V, F = meshgen.icosphere(3, 1.0, 1e-3, 1)
        depth = 5
    else:
        V, F = meshgen.double_sheet(12, 0.05, 5, 0.5, 1e-6, 4)
        depth = 5
    o = oracle.Hierarchy(V, F, depth)
    area = _tri_areas(V, F)
    rng = np.random.default_rng(3)
    w = rng.uniform(0.2, 3.0, size=F.shape[0])
    for d in (o.min_depth, depth):
        Mw = o.mass_weighted(d, w)
        assert abs(Mw.sum() - (w * area).sum()) <= 1e-12 * (w * area).sum()
        for T in rng.integers(0, F.shape[0], size=4):
            e = np.zeros(F.shape[0])
            e[T] = 1.0
            assert abs(o.mass_weighted(d, e).sum() - area[T]) <= 1e-11 * area[T]


def test_weighted_mass_unit_weights_scaling_and_linearity(icosphere):
    """Unit weights give the mass matrix itself; weight 4 everywhere is the mass matrix of the
    surface scaled by 2 (built from scratch: area scales by 4, the grid-unit geometry does not
    change); the weighted mass is linear in the weights."""
    V, F = icosphere
    o = oracle.Hierarchy(V, F, 4)
    o2 = oracle.Hierarchy(2.0 * V, F, 4)
    rng = np.random.default_rng(5)
    w1 = rng.uniform(0, 1, size=F.shape[0])
    w2 = rng.uniform(0, 1, size=F.shape[0])
    for d in range(o.min_depth, o.depth + 1):
        M, _ = o.matrices(d)
        assert abs(o.mass_weighted(d, np.ones(F.shape[0])) - M).max() == 0
        M2, _ = o2.matrices(d)
        assert abs(o.mass_weighted(d, np.full(F.shape[0], 4.0)) - M2).max() <= 1e-14 * abs(M2).max()
        lin = o.mass_weighted(d, w1 + 2 * w2) - o.mass_weighted(d, w1) - 2 * o.mass_weighted(d, w2)
        assert abs(lin).max() <= 1e-14 * abs(M).max()


def test_weighted_rhs_against_weighted_mass(icosphere):
    """For f = 1 the weighted projection is the row sums of the weighted mass matrix (the
    split functions sum to one), two separately written quadratures; unit weights give the
    plain projection, and the total is sum_T w_T int_T f."""
    V, F = icosphere
    o = oracle.Hierarchy(V, F, 4)
    rng = np.random.default_rng(9)
    w = rng.uniform(0.2, 3.0, size=F.shape[0])
    ones = np.ones((V.shape[0], 1))
    r1 = o.project_rhs_weighted(ones, w)[:, 0]
    Mw = o.mass_weighted(o.depth, w)
    assert abs(r1 - np.asarray(Mw.sum(axis=1)).ravel()).max() <= 1e-13 * abs(r1).max()
    f = rng.uniform(-1, 1, size=(V.shape[0], 2))
    assert abs(o.project_rhs_weighted(f, np.ones(F.shape[0])) - o.project_rhs(f)).max() == 0
    # f linear per triangle: int_T f = |T| * mean of its three vertex values
    area = _tri_areas(V, F)
    tot = (w[:, None] * area[:, None] * f[F].mean(axis=1)).sum(axis=0)
    assert np.allclose(o.project_rhs_weighted(f, w).sum(axis=0), tot, rtol=1e-12, atol=1e-14)


def test_weighted_mass_nests(sphere_h, icosphere):
    """The split spaces nest (Claim, Section 4.1), whatever the metric: with per-triangle area
    weights the coarse mass matrix is still P^T M_w P of the finer one."""
    V, F = icosphere
    w = np.random.default_rng(21).uniform(0.25, 4.0, size=F.shape[0])
    for d in range(sphere_h.min_depth + 1, sphere_h.depth + 1):
        P = sphere_h.prolongation(d)
        Mc = sphere_h.mass_weighted(d - 1, w)
        assert abs(P.T @ sphere_h.mass_weighted(d, w) @ P - Mc).max() <= 1e-13 * abs(Mc).max()


def test_cmcf_steps_shrink_the_sphere_by_the_closed_form(icosphere):
    """On a unit sphere the coordinates are eigenfunctions of the Laplacian with eigenvalue 2
    and M_t = r_t^2 M_0, so a cMCF step (Section 5.3) maps radius r to r^3 / (r^2 + 2 delta),
    keeping the centre and the roundness.  The discrete space tracks this to about 0.3 % per
    step; an unweighted right-hand side, inverted weights or weighted stiffness miss by 2-20 %."""
    V, F = icosphere
    o = oracle.Hierarchy(V, F, 5)
    delta = 0.05
    X = V.copy()
    r = np.linalg.norm(X, axis=1).mean()
    for _ in range(3):
        X = o.cmcf_step(X, delta)
        radii = np.linalg.norm(X, axis=1)
        r_new = radii.mean()
        assert abs(r_new / r - r * r / (r * r + 2 * delta)) <= 0.01 * (r * r / (r * r + 2 * delta))
        assert radii.std() <= 1e-3 * r_new
        assert np.abs(X.mean(axis=0)).max() <= 1e-3 * r_new
        r = r_new


def test_spectrum_falls_with_depth_on_nested_spaces(icosphere):
    """The split spaces nest (Claim, Section 4.1), so by the min-max principle each eigenvalue
    of L x = lambda M x can only fall as the depth grows; on the unit sphere the error against
    l(l+1) shrinks with depth (the resolution study of Section 5.1)."""
    V, F = icosphere
    exact = np.array([0.0] + [2.0] * 3 + [6.0] * 5 + [12.0] * 7)
    prev, prev_err = None, None
    for d in (2, 3, 4):
        h = oracle.Hierarchy(V, F, d, min_depth=d)
        M, L = h.matrices(d)
        w = sla.eigh(L.toarray(), M.toarray(), eigvals_only=True, subset_by_index=[0, 15])
        err = np.abs(w[1:] - exact[1:]).max()
        if prev is not None:
            assert np.all(w <= prev + 1e-8 * np.abs(prev).max())
            assert err < 0.6 * prev_err
        prev, prev_err = w, err
