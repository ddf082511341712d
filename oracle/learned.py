"""FP64 oracle of the learned smoother (numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests, the smoke check
and the benchmark's CPU leg use it; it shares no code with the GPU library.

The paper's smoother is Gauss-Seidel (Sections 4.3 and 5.2).  The learned
variant keeps the coloured Gauss-Seidel sweep and lets a small network choose a
relaxation weight per node from that node's stencil:

    x_i <- x_i + omega_i (b_i - sum_j a_ij x_j) / a_ii,   colours 0..7 in turn,

with omega_i = 1.45 + 0.45 y_i / (1 + |y_i|) in (1, 1.9), y = MLP(features_i):
the network may only over-relax.  Because every omega_i lies in (0, 2) the
sweep still converges for any SPD matrix, and omega = 1 is the plain sweep.
The correction of node i is thus a function of its stencil coefficients and
its residual.

Features of node i (28): for each neighbour offset o = corner_j - corner_i in
{-1,0,1}^3, the sum of a_ij / a_ii over the row's entries with that offset
(27 bins; the centre bin, which holds only the diagonal, is replaced by
a_ii / mean_k a_kk), and the row's entry count / 27.

Network: 28 -> 64 (ReLU) -> 1.  Loss over residual samples r0 (columns):
mean_s ||r_s||^2 / ||r0_s||^2, where r is the residual after one V-cycle on the
error equation A e = r0 whose finest-level sweeps (nu1 forward, nu2 backward
colour sweeps) use the learned weights and whose coarse correction is the plain
V-cycle below (coloured Gauss-Seidel, exact dense solve of A + eps I at the
coarsest level, eps = 1e-12 mean diag).  Every step is linear in r, so the
gradient is the exact adjoint: colour steps in reverse, and for the coarse
correction r <- r - A P V_c P^T r the transpose g <- g - P V_c P^T A g (V_c is
symmetric because its sweeps mirror each other).  Residual samples come from the
histories of plain V-cycles.
"""
from __future__ import annotations

import numpy as np

N_FEATURES = 28
HIDDEN = 64


def colours(corner):
    return (corner[:, 0] & 1) | ((corner[:, 1] & 1) << 1) | ((corner[:, 2] & 1) << 2)


def stencil_features(A, corner):
    """Per-node features from a CSR matrix A (scipy) and each dof's grid corner."""
    A = A.tocsr()
    n = A.shape[0]
    diag = A.diagonal()
    X = np.zeros((n, N_FEATURES))
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    off = corner[A.indices] - corner[rows] + 1          # in {0,1,2}^3
    assert off.min() >= 0 and off.max() <= 2
    b = (off[:, 0] * 3 + off[:, 1]) * 3 + off[:, 2]
    np.add.at(X, (rows, b), A.data / diag[rows])
    X[:, 13] = diag / diag.mean()
    X[:, 27] = np.diff(A.indptr) / 27.0
    return X


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
    return 1.45 + 0.45 * y / (1.0 + np.abs(y))


def domega_dy(y):
    return 0.45 / (1.0 + np.abs(y)) ** 2


def sweep_residuals(A, col, omega, R0):
    """Residual form of one coloured sweep with weights omega on A e = r0.
    Returns the list [r^(0), ..., r^(8)] (each n x s)."""
    A = A.tocsr()
    d = A.diagonal()
    rs = [R0.copy()]
    r = R0.copy()
    for c in range(8):
        rows = np.where(col == c)[0]
        delta = (omega[rows] / d[rows])[:, None] * r[rows]
        r = r - A[:, rows] @ delta
        rs.append(r)
    return rs


def loss(A, col, omega, R0):
    r8 = sweep_residuals(A, col, omega, R0)[-1]
    return float(np.mean((r8 ** 2).sum(0) / (R0 ** 2).sum(0)))


def loss_grad_omega(A, col, omega, R0):
    """(loss, dloss/domega) by the reverse of the sweep: for colour c (reversed),
    with g the gradient w.r.t. r^(c+1):  dL/domega_i = -(A g)_i . r^(c)_i / a_ii for
    rows i of colour c, and g <- g - P_c Omega D^-1 (A g)."""
    A = A.tocsr()
    d = A.diagonal()
    rs = sweep_residuals(A, col, omega, R0)
    s = R0.shape[1]
    w = 1.0 / (s * (R0 ** 2).sum(0))                    # per-sample weight of ||r8||^2
    L = float(((rs[-1] ** 2).sum(0) * w).sum())
    g = 2.0 * rs[-1] * w[None, :]
    dom = np.zeros_like(omega)
    for c in range(7, -1, -1):
        rows = np.where(col == c)[0]
        Ag = (A[rows] @ g)                                # rows of colour c of A g (A symmetric)
        dom[rows] = -(Ag * rs[c][rows]).sum(1) / d[rows]
        g = g.copy()
        g[rows] -= (omega[rows] / d[rows])[:, None] * Ag
    return L, dom


def loss_and_grads(p, X, A, col, R0):
    """Loss and gradients w.r.t. every network parameter (FP64, analytic)."""
    Z, H, y = mlp_forward(p, X)
    om = omega_of(y)
    L, dom = loss_grad_omega(A, col, om, R0)
    gy = dom * domega_dy(y)
    grads = {
        "w2": H.T @ gy,
        "b2": np.array([gy.sum()]),
    }
    gH = np.outer(gy, p["w2"]) * (Z > 0)
    grads["W1"] = X.T @ gH
    grads["b1"] = gH.sum(0)
    return L, grads


class Levels:
    """The plain multigrid below the finest level: matrices A_d (scipy CSR), colours
    and prolongations P_d (n_d x n_{d-1}), levels d0..D indexed by depth."""

    def __init__(self, A, col, P, d0, D, nu1=2, nu2=2):
        self.A, self.col, self.P, self.d0, self.D, self.nu1, self.nu2 = A, col, P, d0, D, nu1, nu2
        A0 = A[d0].toarray()
        A0 = A0 + 1e-12 * np.mean(np.diag(A0)) * np.eye(A0.shape[0])
        self.A0inv = np.linalg.inv(A0)

    def sweep(self, d, b, x, order):
        A, col = self.A[d], self.col[d]
        dg = A.diagonal()
        for c in order:
            rows = np.where(col == c)[0]
            x[rows] += (b[rows] - A[rows] @ x) / dg[rows, None]

    def vcycle(self, d, b):
        """Plain V-cycle on A_d x = b from x = 0 (symmetric linear operator of b)."""
        if d == self.d0:
            return self.A0inv @ b
        x = np.zeros_like(b)
        for _ in range(self.nu1):
            self.sweep(d, b, x, range(8))
        r = b - self.A[d] @ x
        P = self.P[d]
        x += P @ self.vcycle(d - 1, P.T @ r)
        for _ in range(self.nu2):
            self.sweep(d, b, x, range(7, -1, -1))
        return x


def cycle_steps(lv):
    steps = []
    for _ in range(lv.nu1):
        steps += [("colour", c) for c in range(8)]
    steps.append(("coarse", None))
    for _ in range(lv.nu2):
        steps += [("colour", c) for c in range(7, -1, -1)]
    return steps


def cycle_loss_grad_omega(lv, omega, R0):
    """Loss and dloss/domega of one V-cycle with learned finest sweeps (residual form)."""
    D = lv.D
    A, col, P = lv.A[D], lv.col[D], lv.P[D]
    dg = A.diagonal()
    steps = cycle_steps(lv)
    rs = [R0.copy()]
    r = R0.copy()
    for kind, c in steps:
        if kind == "colour":
            rows = np.where(col == c)[0]
            delta = np.zeros_like(r)
            delta[rows] = (omega[rows] / dg[rows])[:, None] * r[rows]
            r = r - A @ delta
        else:
            r = r - A @ (P @ lv.vcycle(D - 1, P.T @ r))
        rs.append(r)
    w = 1.0 / (R0.shape[1] * (R0 ** 2).sum(0))
    L = float(((r ** 2).sum(0) * w).sum())
    g = 2.0 * r * w[None, :]
    dom = np.zeros_like(omega)
    for s in range(len(steps) - 1, -1, -1):
        kind, c = steps[s]
        if kind == "colour":
            rows = np.where(col == c)[0]
            Ag = A[rows] @ g
            dom[rows] += -(Ag * rs[s][rows]).sum(1) / dg[rows]
            g = g.copy()
            g[rows] -= (omega[rows] / dg[rows])[:, None] * Ag
        else:
            g = g - P @ lv.vcycle(D - 1, P.T @ (A @ g))
    return L, dom


def cycle_loss_and_grads(p, X, lv, R0):
    Z, H, y = mlp_forward(p, X)
    om = omega_of(y)
    L, dom = cycle_loss_grad_omega(lv, om, R0)
    gy = dom * domega_dy(y)
    grads = {"w2": H.T @ gy, "b2": np.array([gy.sum()])}
    gH = np.outer(gy, p["w2"]) * (Z > 0)
    grads["W1"] = X.T @ gH
    grads["b1"] = gH.sum(0)
    return L, grads


def adam_train(p, X, A, col, samples, steps=200, lr=1e-2, seed=0, batch=8):
    """Reference training loop (Adam on the loss above); returns params and loss history."""
    rng = np.random.default_rng(seed)
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    hist = []
    b1, b2, eps = 0.9, 0.999, 1e-8
    for t in range(1, steps + 1):
        idx = rng.choice(samples.shape[1], size=min(batch, samples.shape[1]), replace=False)
        L, g = loss_and_grads(p, X, A, col, samples[:, idx])
        hist.append(L)
        for k in p:
            m[k] = b1 * m[k] + (1 - b1) * g[k]
            v[k] = b2 * v[k] + (1 - b2) * g[k] ** 2
            mh = m[k] / (1 - b1 ** t)
            vh = v[k] / (1 - b2 ** t)
            p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p, hist
