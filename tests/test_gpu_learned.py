"""Learned relaxation weights (not in the paper): GPU loss and gradient against the
FP64 oracle, training on plain V-cycle residual histories, and what the trained
weights gain over plain Gauss-Seidel on a held-out right-hand side.

Tolerances: the GPU network sees BF16 inputs and weights and accumulates in
FP32; the oracle is given the same BF16-rounded features and first-layer
weights, so the remaining differences are FP32 accumulation (~1e-6 relative in
omega, hence in the loss) and the BF16 rounding of dL/dZ in the tensor-core
product for dW1 (~1e-2 relative); the cycle itself is FP64 on both sides."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import oracle
import paper_1505_03615_gb300 as L
from oracle import learned as LS
from tests._match import permutation

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")
DEV = "cuda:0"


def _bf16(a):
    return torch.tensor(np.asarray(a, dtype=np.float64)).to(torch.bfloat16).double().numpy()


def _flat(p):
    W1 = np.zeros((32, 64))
    W1[:28] = p["W1"]
    return np.concatenate([W1.ravel(), p["b1"], p["w2"], p["b2"]])


def _setup(V, F, depth, d0, t):
    h = L.lbmg_build_hierarchy(V, F, depth, min_depth=d0)
    L.lbmg_assemble(h, t)
    o = oracle.Hierarchy(V, F, depth, min_depth=d0)
    A, col, P = {}, {}, {}
    for d in o.levels():
        M, Lm = o.matrices(d)
        A[d] = (M + t * Lm).tocsr()
        c, _ = o.dofs(d)
        col[d] = LS.colours(c)
        if d > o.min_depth:
            P[d] = o.prolongation(d).tocsr()
    lv = LS.Levels(A, col, P, o.min_depth, depth)
    c, m = L.lbmg_get_dofs(h, depth)
    oc, om = o.dofs(depth)
    perm = permutation(c, m, oc, om, F.shape[0])
    return h, o, lv, perm, oc


def test_learned_loss_and_gradient_match_oracle():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    h, o, lv, perm, oc = _setup(V, F, 4, 2, 1e-2)
    try:
        p = LS.init_params(3, scale=0.3)
        p["W1"] = _bf16(p["W1"])
        p["b2"] = np.array([0.2])
        L.lbmg_learned_params(h, _flat(p))
        n = len(perm)
        rng = np.random.default_rng(1)
        r0 = rng.normal(size=(n, 2))                     # library order
        loss, g = L.lbmg_learned_loss_grad(h, torch.tensor(r0, device=DEV))
        r0o = np.zeros_like(r0)
        r0o[perm] = r0
        X = _bf16(LS.stencil_features(lv.A[4], oc))
        Lo, go = LS.cycle_loss_and_grads(p, X, lv, r0o)
        assert loss == pytest.approx(Lo, rel=1e-5)
        gW1 = g[:32 * 64].reshape(32, 64)
        assert np.abs(gW1[28:]).max() == 0
        rel = lambda a, b: np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)
        assert rel(gW1[:28], go["W1"]) < 2e-2
        assert rel(g[32 * 64:32 * 64 + 64], go["b1"]) < 1e-3
        assert rel(g[32 * 64 + 64:32 * 64 + 128], go["w2"]) < 1e-3
        assert g[-1] == pytest.approx(go["b2"][0], rel=1e-3)
    finally:
        L.lbmg_destroy(h)


def test_training_lowers_the_loss_and_the_learned_solve_stays_exact():
    V, F = meshgen.torus_knot_tube(2, 3, 1.0, 0.06, 200, 20, 1e-6, 3)
    depth, t = 6, 1e-3
    h = L.lbmg_build_hierarchy(V, F, depth, min_depth=2, persistent=1)   # learned weights need the persistent solve
    try:
        L.lbmg_assemble(h, t)
        n = L.lbmg_level_info(h, depth)[0]
        rng = np.random.default_rng(7)
        # residual histories of plain V-cycles on four random right-hand sides
        f = rng.uniform(-1, 1, size=(V.shape[0], 4))
        rhs = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
        L.lbmg_project_rhs(h, torch.tensor(f, device=DEV), rhs)
        L.lbmg_learned_collect(h, rhs, 3, 20)
        p = LS.init_params(0, scale=0.05)
        p["w2"][:] = 0.0
        p["b2"] = np.array([-8.0])                        # start near the plain sweep (omega ~ 1.05)
        L.lbmg_learned_params(h, _flat(p))
        order = rng.integers(0, 80, size=(150, 4))
        hist = L.lbmg_learned_train(h, order, 2e-3)
        assert np.mean(hist[-20:]) < hist[0]
        # held-out right-hand side: vertex y coordinate
        b = torch.zeros((n, 1), dtype=torch.float64, device=DEV)
        L.lbmg_project_rhs(h, torch.tensor(V[:, 1:2].copy(), device=DEV), b)
        res = {}
        for name, on in (("plain", False), ("learned", True)):
            L.lbmg_learned_enable(h, on)
            x = torch.zeros_like(b)
            L.lbmg_solve(h, b, x, 1e-6, 3000, L.LBMG_MIXED)     # warm-up
            x.zero_()
            code, st = L.lbmg_solve(h, b, x, 1e-6, 3000, L.LBMG_MIXED)
            assert code == L.LBMG_OK and st.converged
            res[name] = (st.cycles, st.ms_total, x.cpu().numpy(), st.learned_fallback)
        om = L.lbmg_learned_omega(h)
        assert om.min() > 1.0 and om.max() < 1.9
        rp, ci, M, Lm = L.lbmg_get_matrix(h, depth)
        Mm = sp.csr_matrix((M, ci, rp), shape=(n, n))
        A = (Mm + t * sp.csr_matrix((Lm, ci, rp), shape=(n, n))).tocsc()
        xd = spla.splu(A).solve(b.cpu().numpy())
        for name in res:
            e = res[name][2] - xd
            err = np.sqrt(np.sum(e * (Mm @ e)) / np.sum(xd * (Mm @ xd)))
            assert err < 1e-5, name
        print(f"\nlearned smoother: plain {res['plain'][0]} cycles {res['plain'][1]:.2f} ms; "
              f"learned {res['learned'][0]} cycles {res['learned'][1]:.2f} ms (fallback {res['learned'][3]})")
        # the fallback keeps the learned solve from costing more than a few cycles over plain
        assert res["learned"][0] <= res["plain"][0] * 1.1 + 2
    finally:
        L.lbmg_destroy(h)
