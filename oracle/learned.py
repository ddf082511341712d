"""FP64 oracle of the learned residual correction (numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests, the smoke check
and the benchmark's CPU leg use it; it shares no code with the GPU library.

The paper has no learned part: its smoother is Gauss-Seidel inside the multigrid
cycle (Sections 4.3 and 5.2), and the solver iterates that cycle on the residual.
The learned variant puts a per-node correction of the current residual in front
of each cycle of that iteration:

    delta_i = omega_i r_i / a_ii        for every right-hand-side column of r
    e       = delta + V (r - A delta)   V: the plain cycle from zero on what is left
    x      <- x + e,   r <- b - A x

which is the plain cycle started from delta instead of zero.  omega_i = 1 + y_i /
(1 + |y_i|) lies in (0, 2), and y = 0 gives the undamped Jacobi step; rows under
the relaxation floor (a_ii <= 1e-20 mean diagonal) take no correction.

y_i comes from a 30 -> 64 (ReLU) -> 1 network of node i's features:
  0..26  for each neighbour offset o = corner_j - corner_i in {-1,0,1}^3, the sum of
         a_ij / a_ii over the row's entries with that offset (the centre bin, which
         holds only the diagonal, is replaced by a_ii / mean_k a_kk);
  27     the row's entry count / 27;
  28     the node's local minimal-residual step: with z = A D^-1 r,
         q_i = sum_k r_ik z_ik / sum_k z_ik^2 (0 where z_i = 0), fed as q / (1 + |q|);
  29     the node's share of the residual energy: e_i = sum_k r_ik^2 and e_bar the
         mean of e, fed as e_i / (e_i + e_bar) (0 when r = 0).
Both residual features are unchanged when r is multiplied by any nonzero number,
so the correction is homogeneous of degree one: delta(s r) = s delta(r).

Loss of one residual sample R (n x s: the s right-hand sides of one solve at one
iteration):  L(R) = log(||C (R - A delta(R))||_F^2 / ||R||_F^2) with C = I - A V: the
logarithm of the residual reduction of one learned iteration, so that the mean over
samples counts iterations (a ratio, unlike its logarithm, would let the samples that
converge slowly outweigh those where the correction gains orders of magnitude).  Its
gradient is the exact adjoint: with R1 the new residual and g = 2 R1 / ||R1||^2,
C^T g = g - V (A g) (V is symmetric: its sweeps mirror each other and its coarse
solve is symmetric), dL/d delta = -A C^T g, dL/d omega_i = sum_k (dL/d delta)_ik
r_ik / a_ii, and dL/dy = dL/d omega / (1 + |y|)^2.  The features depend on R only,
so no gradient flows through them.

Acceptance rule of a solve: once an iteration with the correction leaves a
larger residual norm than the iteration before it in some column, the solve
drops the correction and runs plain cycles from then on.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 30
N_STENCIL = 28
HIDDEN = 64
FLOOR = 1e-20


def colours(corner):
    return (corner[:, 0] & 1) | ((corner[:, 1] & 1) << 1) | ((corner[:, 2] & 1) << 2)


def inverse_diagonal(A):
    """1 / a_ii, and 0 on rows under the relaxation floor."""
    d = A.diagonal()
    keep = d > FLOOR * d.mean()
    return np.where(keep, 1.0 / np.where(keep, d, 1.0), 0.0)


def stencil_features(A, corner):
    """Columns 0..27 from a CSR matrix A (scipy) and each dof's grid corner."""
    A = A.tocsr()
    n = A.shape[0]
    diag = A.diagonal()
    X = np.zeros((n, N_STENCIL))
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    off = corner[A.indices] - corner[rows] + 1          # in {0,1,2}^3
    assert off.min() >= 0 and off.max() <= 2
    b = (off[:, 0] * 3 + off[:, 1]) * 3 + off[:, 2]
    np.add.at(X, (rows, b), A.data / diag[rows])
    X[:, 13] = diag / diag.mean()
    X[:, 27] = np.diff(A.indptr) / 27.0
    return X


def residual_features(A, dinv, R):
    """Columns 28, 29 for the residual R (n x s)."""
    R = np.asarray(R, dtype=np.float64).reshape(A.shape[0], -1)
    Z = A @ (dinv[:, None] * R)
    zz = (Z * Z).sum(1)
    q = np.where(zz > 0, (R * Z).sum(1) / np.where(zz > 0, zz, 1.0), 0.0)
    e = (R * R).sum(1)
    ebar = e.mean()
    share = e / (e + ebar) if ebar > 0 else np.zeros_like(e)
    return np.stack([q / (1.0 + np.abs(q)), share], 1)


def features(Xs, A, dinv, R):
    return np.concatenate([Xs, residual_features(A, dinv, R)], 1)


def init_params(seed=0, scale=0.1):
    rng = np.random.default_rng(seed)
    return {
        "W1": rng.normal(0, scale, size=(N_FEATURES, HIDDEN)),
        "b1": np.zeros(HIDDEN),
        "w2": rng.normal(0, scale, size=HIDDEN),
        "b2": np.zeros(1),
    }


def mlp_forward(p, X):
    Z = X @ p["W1"] + p["b1"]
    H = np.maximum(Z, 0.0)
    y = H @ p["w2"] + p["b2"][0]
    return Z, H, y


def omega_of(y):
    return 1.0 + y / (1.0 + np.abs(y))


def domega_dy(y):
    return 1.0 / (1.0 + np.abs(y)) ** 2


def correction(p, Xs, A, dinv, R, feature_map=None):
    """(delta, omega) for the residual R.  feature_map (optional) is applied to the feature
    matrix first: the rounding a low-precision network input applies."""
    R = np.asarray(R, dtype=np.float64).reshape(A.shape[0], -1)
    X = features(Xs, A, dinv, R)
    _, _, y = mlp_forward(p, X if feature_map is None else feature_map(X))
    om = omega_of(y)
    return (om * dinv)[:, None] * R, om


def loss_of_omega(A, dinv, omega, R, vcycle):
    """L for a given omega (the map omega -> L that the gradient differentiates)."""
    D = (omega * dinv)[:, None] * R
    r1 = R - A @ D
    R1 = r1 - A @ vcycle(r1)
    return float(np.log((R1 ** 2).sum() / (R ** 2).sum()))


def loss_grad_omega(A, dinv, omega, R, vcycle):
    """(L, dL/domega) by the adjoint of the learned iteration."""
    U = dinv[:, None] * R
    r1 = R - A @ ((omega[:, None]) * U)
    R1 = r1 - A @ vcycle(r1)
    n1 = (R1 ** 2).sum()
    L = float(np.log(n1 / (R ** 2).sum()))
    g = 2.0 * R1 / n1
    ctg = g - vcycle(A @ g)
    dD = -(A @ ctg)
    return L, (dD * U).sum(1)


def loss_and_grads(p, Xs, A, dinv, R, vcycle, feature_map=None):
    """Loss of one sample and its gradient w.r.t. every network parameter (feature_map as in
    correction)."""
    R = np.asarray(R, dtype=np.float64).reshape(A.shape[0], -1)
    X = features(Xs, A, dinv, R)
    if feature_map is not None:
        X = feature_map(X)
    Z, H, y = mlp_forward(p, X)
    L, dom = loss_grad_omega(A, dinv, omega_of(y), R, vcycle)
    gy = dom * domega_dy(y)
    grads = {"w2": H.T @ gy, "b2": np.array([gy.sum()])}
    gH = np.outer(gy, p["w2"]) * (Z > 0)
    grads["W1"] = X.T @ gH
    grads["b1"] = gH.sum(0)
    return L, grads


def adam_train(p, problems, order, lr=1e-2):
    """Adam over residual samples.  problems[k] = (Xs, A, dinv, vcycle); order is a list of
    steps, each a list of (problem index, sample array); the step's gradient is the mean over
    its samples.  Returns the parameters and the loss history (mean loss per step)."""
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    b1, b2, eps = 0.9, 0.999, 1e-8
    hist = []
    for t, step in enumerate(order, start=1):
        gsum = {k: np.zeros_like(val) for k, val in p.items()}
        lsum = 0.0
        for k, R in step:
            Xs, A, dinv, vc = problems[k]
            L, g = loss_and_grads(p, Xs, A, dinv, R, vc)
            lsum += L
            for q in p:
                gsum[q] += g[q] / len(step)
        hist.append(lsum / len(step))
        for q in p:
            m[q] = b1 * m[q] + (1 - b1) * gsum[q]
            v[q] = b2 * v[q] + (1 - b2) * gsum[q] ** 2
            p[q] = p[q] - lr * (m[q] / (1 - b1 ** t)) / (np.sqrt(v[q] / (1 - b2 ** t)) + eps)
    return p, hist


def corrector(p, Xs, A, dinv):
    """The learned correction as a function of the residual."""
    return lambda r: correction(p, Xs, A, dinv, r)[0]


def solve(corr, A, b, vcycle, tol, max_cycles, x0=None):
    """Defect correction with corr(r) (a correction of the residual, or None for the plain
    iteration) in front of every cycle and the acceptance rule above.  Returns (x, cycles,
    dropped): dropped is the iteration after which the correction was dropped (0 if never)."""
    b = np.asarray(b, dtype=np.float64).reshape(A.shape[0], -1)
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.float64).reshape(b.shape)
    nb2 = (b ** 2).sum(0)
    r = b - A @ x

    def rel(r):
        return np.sqrt((r ** 2).sum(0) / np.where(nb2 > 0, nb2, 1.0))

    prev = rel(r)
    on, dropped = corr is not None, 0
    for k in range(1, max_cycles + 1):
        d = corr(r) if on else np.zeros_like(r)
        x = x + d + vcycle(r - A @ d)
        r = b - A @ x
        cur = rel(r)
        if on and (cur > prev).any():
            on, dropped = False, k
        prev = cur
        if (cur <= tol).all():
            return x, k, dropped
    return x, max_cycles, dropped


def bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64: the rounding the
    tensor-core layer applies to its inputs and weights."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = ((u + 0x7FFF + lsb) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
