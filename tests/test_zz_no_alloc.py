"""The allocation-free residual-norm entry point, checked against lbmg_residual.

lbmg_residual_norms_noalloc serves callers that cannot allocate device memory
while they run (a time-critical loop that cannot afford cudaMalloc's implicit
device synchronisation or an out-of-memory failure midway, a plug-in whose host
application owns the device memory budget).  Its only scratch, the partial sums
of the reduction, is a file-scope device array shared by every call.  Two calls
in a row, on different levels and numbers of right-hand sides, must each match
the norms of lbmg_residual's output to the FP64 parity tolerance (1e-12).
This file is collected last so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

import meshgen
import paper_1505_03615_gb300 as L

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_noalloc_residual_norms_match_the_residual_entry_point():
    V, F = meshgen.icosphere(3, 1.0, 1e-3, 1)
    h = L.lbmg_build_hierarchy(V, F, 5)
    try:
        L.lbmg_assemble(h, 1e-3)
        d0, D = L.lbmg_levels(h)
        rng = np.random.default_rng(21)
        for call, (d, nrhs) in enumerate(((D, 3), (D - 1, 1))):
            n = L.lbmg_level_info(h, d)[0]
            b = torch.tensor(rng.normal(size=(n, nrhs)), device="cuda:0")
            x = torch.tensor(rng.normal(size=(n, nrhs)), device="cuda:0")
            norms = torch.full((nrhs,), float("nan"), dtype=torch.float64, device="cuda:0")
            L.lbmg_residual_norms_noalloc(h, d, b, x, norms)
            r = torch.zeros_like(b)
            L.lbmg_residual(h, d, b, x, r)
            ref = torch.linalg.norm(r, dim=0)
            torch.cuda.synchronize()
            assert torch.allclose(norms, ref, rtol=1e-12, atol=0), (call, norms, ref)
        # the defining property: after the first call (which looks up the scratch array's
        # address), further calls leave the device's free memory exactly as it was
        n = L.lbmg_level_info(h, D)[0]
        b = torch.tensor(rng.normal(size=(n, 3)), device="cuda:0")
        x = torch.tensor(rng.normal(size=(n, 3)), device="cuda:0")
        norms = torch.zeros(3, dtype=torch.float64, device="cuda:0")
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for _ in range(50):
            L.lbmg_residual_norms_noalloc(h, D, b, x, norms)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0
        # more right-hand sides than the scratch holds are refused before any launch
        n = L.lbmg_level_info(h, D)[0]
        b5 = torch.zeros((n, 5), dtype=torch.float64, device="cuda:0")
        out5 = torch.zeros(5, dtype=torch.float64, device="cuda:0")
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_residual_norms_noalloc(h, D, b5, b5, out5)
        assert e.value.code == 1
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_residual_norms_noalloc(h, D + 1, b, x, norms)
        assert e.value.code == 1
    finally:
        L.lbmg_destroy(h)


def test_noalloc_before_assembly_reports_not_assembled():
    V, F = meshgen.icosphere(2, 1.0, 1e-3, 1)
    h = L.lbmg_build_hierarchy(V, F, 4)
    try:
        n = L.lbmg_level_info(h, 4)[0]
        b = torch.zeros((n, 1), dtype=torch.float64, device="cuda:0")
        norms = torch.zeros(1, dtype=torch.float64, device="cuda:0")
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_residual_norms_noalloc(h, 4, b, b, norms)
        assert e.value.code == 5
    finally:
        L.lbmg_destroy(h)
