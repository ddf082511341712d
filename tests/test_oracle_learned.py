"""Pins of the learned-correction oracle (oracle/learned.py) against what the
mathematics fixes, chosen so that a dropped term, a wrong sign or a transposed
operand in it fails one of them:

- the features on hand-made matrices (stencil bins, the local minimal-residual step,
  the residual-energy share), computed by hand;
- the network with zero weights gives omega = 1, the undamped Jacobi step;
- the learned iteration is the plain cycle started from delta (the affine property
  of a linear stationary cycle), checked against the oracle's cycle with a nonzero
  start, an independent code path;
- homogeneity: delta(s r) = s delta(r) for positive, negative, tiny and huge s;
- analytic gradients (w.r.t. omega and every network parameter) against central
  finite differences;
- the acceptance rule drops a correction that makes a residual grow, and the
  learned solve then still converges to the solution.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import meshgen
import oracle
from oracle import learned as LS

T = 1e-2


@pytest.fixture(scope="module")
def system():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    h = oracle.Hierarchy(V, F, 4, min_depth=2)
    M, L = h.matrices(4)
    A = (M + T * L).tocsr()
    corner, _ = h.dofs(4)
    dinv = LS.inverse_diagonal(A)
    Xs = LS.stencil_features(A, corner)

    def vcycle(B):
        B = np.asarray(B).reshape(A.shape[0], -1)
        return h.cycles(T, B, np.zeros_like(B), cycles=1, coloured=True)

    return h, A, dinv, Xs, vcycle, V


def test_stencil_features_follow_definition():
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


def test_residual_features_by_hand():
    # A = [[2,1],[1,2]], r = (1, 0): D^-1 r = (1/2, 0), z = A D^-1 r = (1, 1/2);
    # q_0 = 1*1 / 1^2 = 1 -> 1/2; q_1 = 0 -> 0.  e = (1, 0), mean 1/2: shares 2/3 and 0
    A = sp.csr_matrix(np.array([[2.0, 1.0], [1.0, 2.0]]))
    f = LS.residual_features(A, LS.inverse_diagonal(A), np.array([1.0, 0.0]))
    assert np.allclose(f, [[0.5, 2.0 / 3.0], [0.0, 0.0]], rtol=0, atol=1e-15)
    # two columns: r = [[1, 2], [-1, 0]]: z = [[1/2, 2], [-1/2, 1]];
    # q_0 = (1/2 + 4) / (1/4 + 4) = 18/17, q_1 = (1/2 + 0) / (1/4 + 1) = 2/5
    # e = (5, 1), mean 3: shares 5/8 and 1/4
    f = LS.residual_features(A, LS.inverse_diagonal(A), np.array([[1.0, 2.0], [-1.0, 0.0]]))
    q = np.array([18 / 17, 2 / 5])
    assert np.allclose(f[:, 0], q / (1 + q), rtol=1e-15)
    assert np.allclose(f[:, 1], [5 / 8, 1 / 4], rtol=1e-15)
    # a diagonal matrix: z = r, so q = 1 everywhere (feature 1/2); r = 0: every feature 0
    D = sp.diags([1.0, 4.0, 9.0]).tocsr()
    f = LS.residual_features(D, LS.inverse_diagonal(D), np.array([[1.0], [-3.0], [0.5]]))
    assert np.allclose(f[:, 0], 0.5)
    assert np.array_equal(LS.residual_features(D, LS.inverse_diagonal(D), np.zeros((3, 2))), np.zeros((3, 2)))


def test_floor_rows_take_no_correction():
    A = sp.csr_matrix(np.array([[1.0, 0.0], [0.0, 1e-30]]))
    dinv = LS.inverse_diagonal(A)
    assert dinv[0] == 1.0 and dinv[1] == 0.0


def test_omega_range_and_zero_network():
    y = np.array([-1e12, -3.0, 0.0, 0.5, 1e12])
    om = LS.omega_of(y)
    assert (om > 0).all() and (om < 2).all() and om[2] == 1.0
    assert om[0] < 1e-11 and 2 - om[-1] < 1e-11


def test_zero_network_gives_the_jacobi_step(system):
    h, A, dinv, Xs, vcycle, V = system
    p = {k: np.zeros_like(v) for k, v in LS.init_params().items()}
    R = np.random.default_rng(1).normal(size=(A.shape[0], 3))
    d, om = LS.correction(p, Xs, A, dinv, R)
    assert np.array_equal(om, np.ones(A.shape[0]))
    assert np.array_equal(d, dinv[:, None] * R)


def test_learned_iteration_is_the_cycle_started_from_delta(system):
    h, A, dinv, Xs, vcycle, V = system
    p = LS.init_params(3, 0.3)
    rng = np.random.default_rng(2)
    R = rng.normal(size=(A.shape[0], 2))
    d, _ = LS.correction(p, Xs, A, dinv, R)
    composed = d + vcycle(R - A @ d)
    started = h.cycles(T, R, d, cycles=1, coloured=True)
    assert np.abs(composed - started).max() <= 1e-10 * np.abs(started).max()
    # and the loss is the residual that iteration leaves
    L, _ = LS.loss_grad_omega(A, dinv, LS.correction(p, Xs, A, dinv, R)[1], R, vcycle)
    R1 = R - A @ started
    assert L == pytest.approx(np.log((R1 ** 2).sum() / (R ** 2).sum()), rel=1e-9)


@pytest.mark.parametrize("s", [-3.7, 1e-6, 2.0, 1e5])
def test_correction_is_homogeneous(system, s):
    h, A, dinv, Xs, vcycle, V = system
    p = LS.init_params(4, 0.5)
    R = np.random.default_rng(3).normal(size=(A.shape[0], 3))
    d1, om1 = LS.correction(p, Xs, A, dinv, R)
    d2, om2 = LS.correction(p, Xs, A, dinv, s * R)
    assert np.allclose(om1, om2, rtol=1e-12, atol=0)
    assert np.allclose(d2, s * d1, rtol=1e-11, atol=1e-300)


def test_omega_gradient_matches_finite_differences(system):
    h, A, dinv, Xs, vcycle, V = system
    rng = np.random.default_rng(5)
    R = rng.normal(size=(A.shape[0], 2))
    om = rng.uniform(0.3, 1.7, size=A.shape[0])
    L, g = LS.loss_grad_omega(A, dinv, om, R, vcycle)
    for i in rng.choice(A.shape[0], 6, replace=False):
        eps = 1e-5
        op, omn = om.copy(), om.copy()
        op[i] += eps
        omn[i] -= eps
        fd = (LS.loss_of_omega(A, dinv, op, R, vcycle) - LS.loss_of_omega(A, dinv, omn, R, vcycle)) / (2 * eps)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1e-3 * np.abs(g).max())


def test_parameter_gradients_match_finite_differences(system):
    h, A, dinv, Xs, vcycle, V = system
    p = LS.init_params(7, 0.3)
    rng = np.random.default_rng(6)
    R = rng.normal(size=(A.shape[0], 3))
    L, g = LS.loss_and_grads(p, Xs, A, dinv, R, vcycle)
    picks = [("b2", (0,)), ("w2", (3,)), ("w2", (40,)), ("b1", (5,)), ("W1", (13, 7)), ("W1", (28, 2)),
             ("W1", (29, 11)), ("W1", (27, 30))]
    for name, idx in picks:
        eps = 1e-6
        pp = {k: v.copy() for k, v in p.items()}
        pm = {k: v.copy() for k, v in p.items()}
        pp[name][idx] += eps
        pm[name][idx] -= eps
        fd = (LS.loss_and_grads(pp, Xs, A, dinv, R, vcycle)[0] - LS.loss_and_grads(pm, Xs, A, dinv, R, vcycle)[0]) / (2 * eps)
        scale = max(abs(g[name][idx]), 1e-3 * max(np.abs(v).max() for v in g.values()))
        assert abs(fd - g[name][idx]) <= 1e-5 * scale, (name, idx, fd, g[name][idx])


def test_training_lowers_the_loss(system):
    h, A, dinv, Xs, vcycle, V = system
    b = h.project_rhs(V)
    x = np.zeros_like(b)
    samples = []
    for k in range(12):
        r = b - A @ x
        if k in (2, 5, 8, 11):
            samples.append(r)
        x = x + vcycle(r)
    p = LS.init_params(0, 0.05)
    order = [[(0, samples[k % 4])] for k in range(60)]
    before = np.mean([LS.loss_and_grads(p, Xs, A, dinv, R, vcycle)[0] for R in samples])
    p, hist = LS.adam_train(p, [(Xs, A, dinv, vcycle)], order, lr=1e-2)
    after = np.mean([LS.loss_and_grads(p, Xs, A, dinv, R, vcycle)[0] for R in samples])
    assert after < before - 0.05   # mean log residual reduction per iteration


def test_acceptance_rule_drops_a_harmful_correction_and_the_solve_converges(system):
    h, A, dinv, Xs, vcycle, V = system
    b = h.project_rhs(V)
    ref = spla.splu(A.tocsc()).solve(b)
    # fifty Jacobi steps at once: the residual grows after the first iteration, the rule drops the
    # correction, and the plain cycles that follow converge
    # (errors in the energy norm: nearly dependent restricted hats leave near-null directions
    # along which a 1e-10 residual still allows a visible pointwise difference)
    def err(x):
        e = x - ref
        return np.sqrt(np.einsum("ij,ij->", e, A @ e) / np.einsum("ij,ij->", ref, A @ ref))

    x, cycles, dropped = LS.solve(lambda r: 50.0 * dinv[:, None] * r, A, b, vcycle, 1e-10, 200)
    assert dropped == 1
    assert err(x) <= 1e-9
    # the zero network is a plain Jacobi pre-step: it keeps the correction and beats plain cycles
    p0 = {k: np.zeros_like(v) for k, v in LS.init_params().items()}
    x0, c0, d0 = LS.solve(LS.corrector(p0, Xs, A, dinv), A, b, vcycle, 1e-10, 200)
    xp, cp, _ = LS.solve(None, A, b, vcycle, 1e-10, 200)
    assert err(x0) <= 1e-9
    assert d0 == 0 and c0 < cp


def test_bf16_rounding_matches_torch():
    """The oracle's BF16 rounding (used to give the oracle the GPU network's input rounding)
    against torch's float32 -> bfloat16 conversion, ties and the subnormal range included."""
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(8)
    a = np.concatenate([rng.normal(size=2000), rng.normal(size=500) * 1e-38, [0.0, -0.0, 1.0, 1.00390625,
                        1.01171875, -3.0078125, 65504.0]]).astype(np.float32)
    want = torch.tensor(a).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(LS.bf16(a), want)
