"""Pins of the oracle's multigrid cycles (V and W, coloured or lexicographic smoothing, the
coarsest level solved or relaxed) against what the mathematics fixes.

- A two-level W-cycle is the V-cycle: its two coarse visits solve the same coarse system.
- A coloured sweep is Gauss-Seidel by colour: since rows of one corner-parity colour never
  couple, one sweep equals, colour by colour, a block Jacobi update of that colour's rows,
  computed here with matrix products.
- A cycle with symmetric smoothing (colours or rows forward, then the reverse) and an exact or
  symmetric coarsest treatment is a symmetric method: its error operator E = I - B A is
  self-adjoint in the A inner product, its eigenvalues are real and lie in [0, 1), and a
  W-cycle contracts at least as much as the V-cycle.
- The solution of the system is a fixed point of every cycle.
"""
import numpy as np
import pytest

import meshgen
import oracle

T = 1e-2


@pytest.fixture(scope="module")
def small():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    return V, F


def _A(h, d):
    M, Lm = h.matrices(d)
    return (M + T * Lm).toarray()


def _error_operator(h, **kw):
    """E with E e = error after one cycle on A x = 0 from x = e, column by column"""
    n = h.ndof(h.depth)
    return h.cycles(T, np.zeros((n, n)), np.eye(n), cycles=1, **kw)


@pytest.mark.parametrize("coloured", [False, True])
def test_two_level_w_cycle_is_the_v_cycle(small, coloured):
    V, F = small
    h = oracle.Hierarchy(V, F, 4, min_depth=3)
    n = h.ndof(4)
    rng = np.random.default_rng(1)
    b = rng.normal(size=(n, 2))
    x0 = rng.normal(size=(n, 2))
    xv = h.cycles(T, b, x0, cycles=2, gamma=1, coloured=coloured)
    xw = h.cycles(T, b, x0, cycles=2, gamma=2, coloured=coloured)
    assert np.array_equal(xv, xw)


def test_coloured_sweep_is_colour_block_jacobi(small):
    """One forward sweep (colours 0..7) and one backward sweep (7..0) against the block form
    x_c <- x_c + D_c^-1 (b - A x)_c applied colour after colour."""
    V, F = small
    h = oracle.Hierarchy(V, F, 3, min_depth=3)   # one level: the coarsest is relaxed
    A = _A(h, 3)
    n = A.shape[0]
    corner, _ = h.dofs(3)
    colour = (corner[:, 0] & 1) + 2 * (corner[:, 1] & 1) + 4 * (corner[:, 2] & 1)
    dg = np.diag(A)
    assert dg.min() > 1e-20 * dg.mean()          # no row falls under the relaxation floor here
    rng = np.random.default_rng(2)
    b = rng.normal(size=n)
    x0 = rng.normal(size=n)
    for nu1, nu2, order in ((1, 0, range(8)), (0, 1, range(7, -1, -1))):
        x = x0.copy()
        for c in order:
            rows = colour == c
            x[rows] += (b - A @ x)[rows] / dg[rows]
        got = h.cycles(T, b, x0, cycles=1, nu1=nu1, nu2=nu2, coloured=True, coarse_smooth=True)[:, 0]
        assert np.abs(got - x).max() <= 1e-13 * np.abs(x).max()


@pytest.mark.parametrize("gamma,coloured,coarse_smooth", [(1, True, False), (2, True, False), (1, False, False),
                                                          (2, True, True)])
def test_cycle_error_operator_is_self_adjoint_in_the_energy_product(small, gamma, coloured, coarse_smooth):
    V, F = small
    h = oracle.Hierarchy(V, F, 4, min_depth=1)
    A = _A(h, 4)
    E = _error_operator(h, gamma=gamma, coloured=coloured, coarse_smooth=coarse_smooth)
    AE = A @ E
    assert np.abs(AE - AE.T).max() <= 1e-10 * np.abs(AE).max()
    lam = np.linalg.eigvals(E)
    assert np.abs(lam.imag).max() <= 1e-8
    assert lam.real.min() >= -1e-9 and lam.real.max() < 1.0


def test_w_cycle_contracts_at_least_as_much_as_the_v_cycle(small):
    V, F = small
    h = oracle.Hierarchy(V, F, 4, min_depth=1)
    rho = {g: np.abs(np.linalg.eigvals(_error_operator(h, gamma=g, coloured=True))).max() for g in (1, 2)}
    assert rho[2] <= rho[1] + 1e-9
    assert rho[1] < 1.0


@pytest.mark.parametrize("gamma,coloured,coarse_smooth", [(1, True, False), (2, True, False), (2, False, True)])
def test_solution_is_a_fixed_point_of_every_cycle(small, gamma, coloured, coarse_smooth):
    V, F = small
    h = oracle.Hierarchy(V, F, 4, min_depth=2)
    A = _A(h, 4)
    rng = np.random.default_rng(3)
    xs = rng.normal(size=(A.shape[0], 2))
    x = h.cycles(T, A @ xs, xs, cycles=3, gamma=gamma, coloured=coloured, coarse_smooth=coarse_smooth)
    assert np.abs(x - xs).max() <= 1e-11 * np.abs(xs).max()


def test_cube_grid_model():
    """The equidistant cubes: closed, consistently oriented cube surfaces, one connected
    component per cube, spaced by the gap."""
    V, F = meshgen.cube_grid(3, size=1.0, gap=1.0, subdiv=2, jitter=0.0)
    assert F.shape[0] == 27 * 12 * 4
    edges = {}
    for t in F:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            edges[(a, b)] = edges.get((a, b), 0) + 1
    assert all(v == 1 for v in edges.values()) and all((b, a) in edges for (a, b) in edges)
    assert V.shape[0] - len(edges) // 2 + F.shape[0] == 2 * 27
    mn = V.reshape(27, -1, 3).min(axis=1)
    assert np.allclose(np.unique(mn[:, 0]), [0.0, 2.0, 4.0])
