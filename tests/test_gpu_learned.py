"""The learned residual correction (not in the paper) through the C-ABI, against the FP64
oracle of oracle/learned.py:

- loss and gradient of one residual sample (the training path);
- omega and delta of the solve path, in FP64 and in mixed precision, including the
  zero network (the plain Jacobi start) and homogeneity under an exact scaling;
- one learned FP64 iteration against the oracle's learned iteration;
- the acceptance test: the device stopping test and the host loop drop the correction at
  the same iteration and return the same iterate.

Tolerances: the GPU network sees BF16 features and first-layer weights and accumulates in
FP32; the oracle is given the same BF16 rounding (oracle.learned.bf16), so what remains is
FP32 accumulation (about 1e-6 in omega, hence in the loss), the BF16 rounding of dL/dZ in the
tensor-core product for dW1 (about 1e-2 relative), and, rarely, a feature that lands on the
other side of a BF16 rounding boundary (FP32 features on the mixed path): such a node's omega
moves by at most a few hundredths, and at most 1% of the nodes may differ by more than 1e-3.
The cycles are FP64 on both sides.  The gain of a trained network is the subject of
tests/test_gpu_learned_gain.py.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import oracle
import paper_1505_03615_gb300 as L
from oracle import learned as LS
from tests._match import permutation

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"
T = 1e-2


def _flat(p):
    W1 = np.zeros((32, 64))
    W1[:30] = p["W1"]
    return np.concatenate([W1.ravel(), p["b1"], p["w2"], p["b2"]])


def _gpu_params(p):
    """the parameters as the GPU holds them: BF16 first layer, FP32 the rest"""
    return {"W1": LS.bf16(p["W1"]), "b1": p["b1"].astype(np.float32).astype(np.float64),
            "w2": p["w2"].astype(np.float32).astype(np.float64), "b2": p["b2"].astype(np.float32).astype(np.float64)}


@pytest.fixture(scope="module")
def pair():
    V, F = meshgen.icosphere(3, 1.0, 1e-3, 1)
    depth, d0 = 5, 2
    h = L.lbmg_build_hierarchy(V, F, depth, min_depth=d0)
    L.lbmg_assemble(h, T)
    o = oracle.Hierarchy(V, F, depth, min_depth=d0)
    M, Lm = o.matrices(depth)
    A = (M + T * Lm).tocsr()
    oc, om = o.dofs(depth)
    c, m = L.lbmg_get_dofs(h, depth)
    perm = permutation(c, m, oc, om, F.shape[0])
    assert (perm >= 0).all()
    dinv = LS.inverse_diagonal(A)
    Xs = LS.stencil_features(A, oc)

    def vcycle(B):
        B = np.asarray(B).reshape(A.shape[0], -1)
        return o.cycles(T, B, np.zeros_like(B), cycles=1, coloured=True)

    # a residual of the plain iteration (oracle order): the projected coordinates after two cycles
    b = o.project_rhs(V)
    x = vcycle(b)
    x = x + vcycle(b - A @ x)
    R = b - A @ x
    yield h, o, A, dinv, Xs, vcycle, perm, R, V
    L.lbmg_destroy(h)


def _to_lib(a, perm):
    return np.ascontiguousarray(a[perm])


def test_loss_and_gradient_match_oracle(pair):
    h, o, A, dinv, Xs, vcycle, perm, R, V = pair
    p = LS.init_params(3, scale=0.3)
    p["b2"] = np.array([0.2])
    L.lbmg_learned_params(h, _flat(p))
    loss, g = L.lbmg_learned_loss_grad(h, torch.tensor(_to_lib(R, perm), device=DEV))
    Lo, go = LS.loss_and_grads(_gpu_params(p), Xs, A, dinv, R, vcycle, feature_map=LS.bf16)
    assert loss == pytest.approx(Lo, rel=1e-5)
    gW1 = g[:32 * 64].reshape(32, 64)
    assert np.abs(gW1[30:]).max() == 0
    rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
    assert rel(gW1[:30], go["W1"]) < 2e-2
    assert rel(g[32 * 64:32 * 64 + 64], go["b1"]) < 1e-3
    assert rel(g[32 * 64 + 64:32 * 64 + 128], go["w2"]) < 1e-3
    assert g[-1] == pytest.approx(go["b2"][0], rel=1e-3)


@pytest.mark.parametrize("precision", [L.LBMG_FP64, L.LBMG_MIXED])
def test_solve_path_correction_matches_oracle(pair, precision):
    h, o, A, dinv, Xs, vcycle, perm, R, V = pair
    p = LS.init_params(11, scale=0.3)
    p["b2"] = np.array([-0.3])
    L.lbmg_learned_params(h, _flat(p))
    n, ns = R.shape
    r = torch.tensor(_to_lib(R, perm), device=DEV)
    om = torch.zeros(n, dtype=torch.float64, device=DEV)
    de = torch.zeros((n, ns), dtype=torch.float64, device=DEV)
    L.lbmg_learned_apply(h, r, precision, om, de)
    d_o, om_o = LS.correction(_gpu_params(p), Xs, A, dinv, R, feature_map=LS.bf16)
    got = om.cpu().numpy()
    diff = np.abs(got - om_o[perm])
    assert diff.max() < 5e-2 and np.mean(diff > 1e-3) < 0.01, (diff.max(), np.mean(diff > 1e-3))
    assert (got > 0).all() and (got < 2).all()
    # delta is omega D^-1 r with the library's own diagonal, in the path's precision
    rp, ci, Mv, Lv = L.lbmg_get_matrix(h, o.depth)
    Al = sp.csr_matrix((Mv + T * Lv, ci, rp), shape=(n, n))
    want = (got * LS.inverse_diagonal(Al))[:, None] * _to_lib(R, perm)
    tol = 1e-13 if precision == L.LBMG_FP64 else 1e-6
    assert np.abs(de.cpu().numpy() - want).max() <= tol * np.abs(want).max()


@pytest.mark.parametrize("precision", [L.LBMG_FP64, L.LBMG_MIXED])
def test_zero_network_and_exact_scaling(pair, precision):
    h, o, A, dinv, Xs, vcycle, perm, R, V = pair
    L.lbmg_learned_params(h, np.zeros(L.lbmg_learned_nparams()))
    n, ns = R.shape
    r = torch.tensor(_to_lib(R, perm), device=DEV)
    om = torch.zeros(n, dtype=torch.float64, device=DEV)
    de = torch.zeros((n, ns), dtype=torch.float64, device=DEV)
    L.lbmg_learned_apply(h, r, precision, om, de)
    assert torch.all(om == 1.0)
    # the plain Jacobi start: delta = D^-1 r in the path's precision
    rp, ci, Mv, Lv = L.lbmg_get_matrix(h, o.depth)
    di = LS.inverse_diagonal(sp.csr_matrix((Mv + T * Lv, ci, rp), shape=(n, n)))
    want = di[:, None] * _to_lib(R, perm)
    tol = 1e-15 if precision == L.LBMG_FP64 else 1e-6
    assert np.abs(de.cpu().numpy() - want).max() <= tol * np.abs(want).max()
    # a power-of-two scaling of r scales delta exactly and leaves omega unchanged
    p = LS.init_params(5, scale=0.4)
    L.lbmg_learned_params(h, _flat(p))
    om2 = torch.zeros_like(om)
    de2 = torch.zeros_like(de)
    L.lbmg_learned_apply(h, r, precision, om, de)
    L.lbmg_learned_apply(h, -4.0 * r, precision, om2, de2)
    assert torch.equal(om, om2)
    assert torch.equal(-4.0 * de, de2)


def test_one_learned_iteration_matches_oracle(pair):
    h, o, A, dinv, Xs, vcycle, perm, R, V = pair
    p = LS.init_params(21, scale=0.3)
    L.lbmg_learned_params(h, _flat(p))
    L.lbmg_learned_enable(h, True)
    try:
        n = R.shape[0]
        rng = np.random.default_rng(4)
        b = A @ rng.normal(size=(n, 3))
        x0 = rng.normal(size=(n, 3))
        x = torch.tensor(_to_lib(x0, perm), device=DEV)
        assert L.lbmg_vcycles(h, torch.tensor(_to_lib(b, perm), device=DEV), x, 1, L.LBMG_FP64) == L.LBMG_OK
        r0 = b - A @ x0
        d, _ = LS.correction(_gpu_params(p), Xs, A, dinv, r0, feature_map=LS.bf16)
        xo = x0 + d + vcycle(r0 - A @ d)
        got = np.zeros_like(x0)
        got[perm] = x.cpu().numpy()

        def energy(v):
            return np.sqrt(np.einsum("ij,ij->j", v, A @ v))
        # omega agrees to ~1e-6 (rare BF16 boundary cases: a few hundredths on single nodes)
        assert (energy(got - xo) <= 1e-4 * energy(xo - x0)).all()
    finally:
        L.lbmg_learned_enable(h, False)


def test_acceptance_test_drops_a_harmful_correction_on_both_loops():
    """A correction that raises the residual is dropped after its first iteration, by the device
    stopping test and by the host loop alike, with bitwise equal iterates.  omega close to 2
    (twice the Jacobi step) in front of cycles without smoothing (nu1 = nu2 = 0) raises the
    residual of a random start by a factor of about two, in the oracle as on the GPU."""
    V, F = meshgen.icosphere(3, 1.0, 1e-3, 1)
    depth, d0, cycles = 5, 2, 6
    h = L.lbmg_build_hierarchy(V, F, depth, min_depth=d0, nu1=0, nu2=0)
    try:
        L.lbmg_assemble(h, T)
        p = {k: np.zeros_like(v) for k, v in LS.init_params().items()}
        p["b2"] = np.array([1e6])
        L.lbmg_learned_params(h, _flat(p))
        L.lbmg_learned_enable(h, True)
        n = L.lbmg_level_info(h, depth)[0]
        x0 = torch.tensor(np.random.default_rng(1).normal(size=(n, 3)), device=DEV)
        b = torch.zeros_like(x0)
        res = {}
        for host in (0, 1):
            L.lbmg_set_host_check(h, host)
            x = x0.clone()
            code, st = L.lbmg_solve(h, b, x, 1e-12, cycles, L.LBMG_MIXED)
            res[host] = (code, st.cycles, st.learned, st.learned_fallback, x)
        assert res[0][:4] == res[1][:4] == (L.LBMG_NOT_CONVERGED, cycles, 1, 1)
        assert torch.equal(res[0][4], res[1][4])
        # the same start in the oracle: the first learned iteration raises the residual
        o = oracle.Hierarchy(V, F, depth, min_depth=d0)
        M, Lm = o.matrices(depth)
        A = (M + T * Lm).tocsr()
        oc, om = o.dofs(depth)
        c, m = L.lbmg_get_dofs(h, depth)
        perm = permutation(c, m, oc, om, F.shape[0])
        xo0 = np.zeros((n, 3))
        xo0[perm] = x0.cpu().numpy()
        vc = lambda B: o.cycles(T, B, np.zeros_like(B), cycles=1, nu1=0, nu2=0, coloured=True)
        corr = LS.corrector(p, LS.stencil_features(A, oc), A, LS.inverse_diagonal(A))
        _, k, dropped = LS.solve(corr, A, np.zeros((n, 3)), vc, 1e-12, cycles, x0=xo0)
        assert dropped == 1 and k == cycles
    finally:
        L.lbmg_destroy(h)
