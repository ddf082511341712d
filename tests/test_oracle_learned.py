"""Pins of the learned-smoother oracle: analytic gradients against central finite
differences, the omega = 1 case against a plain coloured Gauss-Seidel sweep, and
features against their definition on a hand-made stencil."""
import numpy as np
import pytest
import scipy.sparse as sp

import meshgen
import oracle
from oracle import learned as LS


@pytest.fixture(scope="module")
def system():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    h = oracle.Hierarchy(V, F, 4, min_depth=4)
    M, L = h.matrices(4)
    A = (M + 1e-2 * L).tocsr()
    corner, _ = h.dofs(4)
    return A, corner


def test_features_follow_definition():
    corner = np.array([[1, 1, 1], [2, 1, 1], [1, 0, 1], [2, 2, 2]])
    A = sp.csr_matrix(np.array([[4.0, -1.0, -2.0, 0.5], [-1.0, 3.0, 0.0, 0.0],
                                [-2.0, 0.0, 5.0, 0.0], [0.5, 0.0, 0.0, 2.0]]))
    X = LS.stencil_features(A, corner)
    mean = np.mean([4.0, 3.0, 5.0, 2.0])
    # row 0: offsets (+1,0,0) -> bin (2*3+1)*3+1 = 22, (0,-1,0) -> bin (1*3+0)*3+1 = 10, (+1,+1,+1) -> 26
    assert X[0, 22] == pytest.approx(-1.0 / 4.0)
    assert X[0, 10] == pytest.approx(-2.0 / 4.0)
    assert X[0, 26] == pytest.approx(0.5 / 4.0)
    assert X[0, 13] == pytest.approx(4.0 / mean)
    assert X[0, 27] == pytest.approx(4 / 27)
    assert X[1, 4] == pytest.approx(-1.0 / 3.0)   # offset (-1,0,0) -> (0*3+1)*3+1 = 4


def test_unit_weights_give_the_plain_coloured_sweep(system):
    A, corner = system
    col = LS.colours(corner)
    rng = np.random.default_rng(0)
    n = A.shape[0]
    b = rng.normal(size=(n, 2))
    # plain coloured GS in x-form from x = 0 on A x = b
    x = np.zeros_like(b)
    d = A.diagonal()
    for c in range(8):
        rows = np.where(col == c)[0]
        x[rows] += (b[rows] - A[rows] @ x) / d[rows, None]
    r8 = LS.sweep_residuals(A, col, np.ones(n), b)[-1]
    assert np.abs(r8 - (b - A @ x)).max() < 1e-12 * np.abs(b).max()


def test_zero_network_gives_the_midpoint_weight():
    p = LS.init_params(0)
    for k in p:
        p[k] = np.zeros_like(p[k])
    X = np.random.default_rng(1).normal(size=(5, LS.N_FEATURES))
    _, _, y = LS.mlp_forward(p, X)
    assert np.all(LS.omega_of(y) == 1.45)


def test_gradients_match_finite_differences(system):
    A, corner = system
    col = LS.colours(corner)
    X = LS.stencil_features(A, corner)
    rng = np.random.default_rng(2)
    R0 = A @ rng.normal(size=(A.shape[0], 3))
    p = LS.init_params(3, scale=0.3)
    L, g = LS.loss_and_grads(p, X, A, col, R0)
    eps = 1e-6
    for key, idxs in (("W1", [(0, 0), (13, 5), (27, 63), (4, 17)]), ("b1", [(3,), (40,)]),
                      ("w2", [(0,), (31,)]), ("b2", [(0,)])):
        for ix in idxs:
            q = {k: v.copy() for k, v in p.items()}
            q[key][ix] += eps
            Lp = LS.loss(A, col, LS.omega_of(LS.mlp_forward(q, X)[2]), R0)
            q[key][ix] -= 2 * eps
            Lm = LS.loss(A, col, LS.omega_of(LS.mlp_forward(q, X)[2]), R0)
            fd = (Lp - Lm) / (2 * eps)
            assert abs(fd - g[key][ix]) <= 1e-6 * max(1e-3, abs(fd)), (key, ix, fd, g[key][ix])
    assert L == pytest.approx(LS.loss(A, col, LS.omega_of(LS.mlp_forward(p, X)[2]), R0), rel=1e-12)


def test_weights_stay_in_convergent_range():
    y = np.linspace(-1e6, 1e6, 1001)
    om = LS.omega_of(y)
    assert om.min() > 1.0 - 1e-12 and om.max() < 1.9 + 1e-12


@pytest.fixture(scope="module")
def levels():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    h = oracle.Hierarchy(V, F, 4, min_depth=2)
    A, col, P = {}, {}, {}
    for d in h.levels():
        M, L = h.matrices(d)
        A[d] = (M + 1e-2 * L).tocsr()
        c, _ = h.dofs(d)
        col[d] = LS.colours(c)
        if d > h.min_depth:
            P[d] = h.prolongation(d).tocsr()
    corner, _ = h.dofs(4)
    return LS.Levels(A, col, P, h.min_depth, 4), corner


def test_coarse_vcycle_is_symmetric(levels):
    lv, _ = levels
    rng = np.random.default_rng(4)
    n = lv.A[3].shape[0]
    u, v = rng.normal(size=(n, 1)), rng.normal(size=(n, 1))
    a, b = (u.T @ lv.vcycle(3, v)).item(), (lv.vcycle(3, u).T @ v).item()
    assert abs(a - b) <= 1e-12 * abs(a)


def test_cycle_loss_with_unit_weights_is_the_plain_vcycle(levels):
    lv, _ = levels
    rng = np.random.default_rng(6)
    A = lv.A[4]
    R0 = rng.normal(size=(A.shape[0], 2))
    L, _ = LS.cycle_loss_grad_omega(lv, np.ones(A.shape[0]), R0)
    r = R0 - A @ lv.vcycle(4, R0)
    expect = np.mean((r ** 2).sum(0) / (R0 ** 2).sum(0))
    assert L == pytest.approx(expect, rel=1e-10)


def test_cycle_gradients_match_finite_differences(levels):
    lv, corner = levels
    A = lv.A[4]
    X = LS.stencil_features(A, corner)
    rng = np.random.default_rng(8)
    R0 = rng.normal(size=(A.shape[0], 2))
    p = LS.init_params(9, scale=0.3)
    L, g = LS.cycle_loss_and_grads(p, X, lv, R0)
    eps = 1e-6
    for key, ix in (("W1", (0, 1)), ("W1", (13, 7)), ("b1", (5,)), ("w2", (2,)), ("b2", (0,))):
        q = {k: v.copy() for k, v in p.items()}
        q[key][ix] += eps
        Lp, _ = LS.cycle_loss_grad_omega(lv, LS.omega_of(LS.mlp_forward(q, X)[2]), R0)
        q[key][ix] -= 2 * eps
        Lm, _ = LS.cycle_loss_grad_omega(lv, LS.omega_of(LS.mlp_forward(q, X)[2]), R0)
        fd = (Lp - Lm) / (2 * eps)
        assert abs(fd - g[key][ix]) <= 1e-5 * max(1e-4, abs(fd)), (key, ix, fd, g[key][ix])
