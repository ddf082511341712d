"""FP64 oracle of the learned smoother (numpy).

TEST INFRASTRUCTURE, like the rest of ``oracle/``: only tests, the smoke check
and the benchmark's CPU leg use it; it shares no code with the GPU library.

The paper's smoother is Gauss-Seidel (Sections 4.3 and 5.2).  The learned
variant keeps the coloured Gauss-Seidel sweep and lets a small network choose a
relaxation weight per node from that node's stencil:

    x_i <- x_i + omega_i (b_i - sum_j a_ij x_j) / a_ii,   colours 0..7 in turn,

with omega_i = 1 + 0.9 y_i / (1 + |y_i|) in (0.1, 1.9), y = MLP(features_i).
Because every omega_i lies in (0, 2) the sweep converges for any SPD matrix,
and omega = 1 is exactly the plain sweep.  The correction of node i is thus a
function of its stencil coefficients and its residual.

Features of node i (28): for each neighbour offset o = corner_j - corner_i in
{-1,0,1}^3, the sum of a_ij / a_ii over the row's entries with that offset
(27 bins; the centre bin, which holds only the diagonal, is replaced by
a_ii / mean_k a_kk), and the row's entry count / 27.

Network: 28 -> 64 (ReLU) -> 1.  Loss over residual samples r0 (columns):
mean_s ||r8_s||^2 / ||r0_s||^2, where r8 is the residual after one learned sweep
applied to the error equation (the residual form of the sweep above).
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
    return 1.0 + 0.9 * y / (1.0 + np.abs(y))


def domega_dy(y):
    return 0.9 / (1.0 + np.abs(y)) ** 2


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
