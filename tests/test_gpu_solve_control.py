"""The solve's stopping test on the device (through the C-ABI).

By default a solve is one CUDA-graph launch: a conditional WHILE node runs one
iteration (V-cycle step or preconditioned CG step) and a one-thread check kernel
that compares the residual norms with the tolerance; the host waits once, for the
final status.  These tests check that the number of host synchronizations does
not grow with the number of cycles, that the device test stops where the host test
(one launch and one norm read per iteration, host_check = 1) stops, with bitwise
the same iterate, and the stopping rule's edge cases on every solve path.
"""
import numpy as np
import pytest

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
DEV = "cuda:0"


@pytest.fixture(scope="module")
def knot():
    V, F = meshgen.torus_knot_tube(2, 3, 1.0, 0.08, 200, 24, 1e-6, 2)
    h = L.lbmg_build_hierarchy(V, F, 6)
    L.lbmg_assemble(h, 1e-3)
    n = L.lbmg_level_info(h, 6)[0]
    rhs = torch.zeros((n, 3), dtype=torch.float64, device=DEV)
    L.lbmg_project_rhs(h, torch.tensor(V, device=DEV), rhs)
    yield h, rhs
    L.lbmg_destroy(h)


@pytest.mark.parametrize("solver", ["vcycle", "pcg"])
@pytest.mark.parametrize("precision", [L.LBMG_MIXED, L.LBMG_FP64])
def test_one_host_synchronization_whatever_the_cycle_count(knot, solver, precision):
    h, rhs = knot
    solve = L.lbmg_solve_pcg if solver == "pcg" else L.lbmg_solve
    runs = {}
    for tol in (1e-3, 1e-9):
        x = torch.zeros_like(rhs)
        code, st = solve(h, rhs, x, tol, 500, precision)
        assert code == L.LBMG_OK and st.converged == 1
        assert max(st.rel_residual[:3]) <= tol
        runs[tol] = st
    assert runs[1e-9].cycles > 2 * runs[1e-3].cycles
    for st in runs.values():
        assert st.host_syncs == 1
    # host output buffers: still one wait (the copy back and the status read together)
    xh = np.zeros((rhs.shape[0], 3))
    code, st = solve(h, rhs.cpu().numpy(), xh, 1e-9, 500, precision)
    assert code == L.LBMG_OK and st.host_syncs == 1


@pytest.mark.parametrize("solver", ["vcycle", "pcg"])
def test_device_stopping_test_matches_host_loop_bitwise(knot, solver):
    h, rhs = knot
    solve = L.lbmg_solve_pcg if solver == "pcg" else L.lbmg_solve
    out = []
    try:
        for host_check in (0, 1):
            L.lbmg_set_host_check(h, host_check)
            x = torch.zeros_like(rhs)
            code, st = solve(h, rhs, x, 1e-8, 500, L.LBMG_MIXED)
            assert code == L.LBMG_OK
            out.append((x.cpu().numpy(), st.cycles, list(st.rel_residual[:3]), st.host_syncs))
    finally:
        L.lbmg_set_host_check(h, 0)
    (xd, cd, rd, sd), (xh, ch, rh, sh) = out
    assert cd == ch and rd == rh
    assert np.array_equal(xd, xh)
    assert sd == 1 and sh >= cd


def test_vcycles_runs_exactly_the_requested_cycles(knot):
    """lbmg_vcycles has no stopping test: k calls of one cycle equal one call of k cycles."""
    h, rhs = knot
    x1 = torch.zeros_like(rhs)
    for _ in range(5):
        L.lbmg_vcycles(h, rhs, x1, 1, L.LBMG_FP64)
    x5 = torch.zeros_like(rhs)
    L.lbmg_vcycles(h, rhs, x5, 5, L.LBMG_FP64)
    assert torch.equal(x1, x5)
    x0 = torch.zeros_like(rhs)
    L.lbmg_vcycles(h, rhs, x0, 0, L.LBMG_FP64)
    assert torch.count_nonzero(x0) == 0


@pytest.mark.parametrize("path", ["vcycle", "pcg", "persistent", "host_check"])
def test_zero_right_hand_side_is_judged_by_the_absolute_residual(path):
    """b = 0 with a nonzero warm start: every path iterates towards x = 0 until ||A x|| <= tol
    (a zero right-hand side used to read as converged before any cycle on the graph and CG
    paths, with x unchanged, while the persistent solve ran to its cycle cap)."""
    V, F = meshgen.icosphere(3, 1.0, 1e-3, 1)
    h = L.lbmg_build_hierarchy(V, F, 5, persistent=int(path == "persistent"), host_check=int(path == "host_check"))
    try:
        L.lbmg_assemble(h, 1e-2)
        n = L.lbmg_level_info(h, 5)[0]
        rhs = torch.zeros((n, 2), dtype=torch.float64, device=DEV)
        x0 = torch.tensor(np.random.default_rng(5).uniform(0, 1, size=(n, 2)), device=DEV)
        r = torch.zeros_like(rhs)
        L.lbmg_residual(h, 5, rhs, x0, r)
        r0_cols = torch.linalg.norm(r, dim=0).cpu().numpy()
        r0 = float(r0_cols.max())
        tol = 1e-6 * r0
        x = x0.clone()
        solve = L.lbmg_solve_pcg if path == "pcg" else L.lbmg_solve
        code, st = solve(h, rhs, x, tol, 500, L.LBMG_FP64)
        assert code == L.LBMG_OK and st.converged == 1 and st.cycles > 0
        L.lbmg_residual(h, 5, rhs, x, r)
        assert float(torch.linalg.norm(r, dim=0).max()) <= tol * (1 + 1e-9)
        # the reported initial residual is the absolute one, ||0 - A x0||
        assert np.allclose(st.initial_residual[:2], r0_cols, rtol=1e-9, atol=0)
    finally:
        L.lbmg_destroy(h)
