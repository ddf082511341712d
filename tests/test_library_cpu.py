"""Host-only checks of the C-ABI library: it builds, loads without a GPU, exports
every entry point declared in include/lbmg.h, and rejects bad input on the host
before touching a device."""
import ctypes as C
import os

import numpy as np
import pytest

import paper_1505_03615_gb300 as L


def test_library_loads_and_exports_every_declared_symbol():
    lib = L.load_library()
    names = L.exported_symbols()
    assert len(names) >= 20
    for name in names:
        assert hasattr(lib, name), name
    # the binding exposes a function of the same name for each entry point
    for name in names:
        assert hasattr(L, name), name


def test_library_is_built_for_sm_103a():
    import subprocess
    from paper_1505_03615_gb300 import build
    path = build.build()
    assert os.path.dirname(path).startswith(os.path.dirname(os.path.abspath(L.__file__)))
    out = subprocess.run(["/usr/local/cuda/bin/cuobjdump", "--list-elf", path], capture_output=True, text=True)
    if out.returncode == 0:
        assert "sm_103a" in out.stdout


def test_status_strings_and_defaults():
    assert L.lbmg_status_string(0) == "ok"
    assert L.lbmg_status_string(4) == "not converged"
    o = L.lbmg_default_options()
    assert (o.min_depth, o.coarse_max, o.nu1, o.nu2, o.split) == (-1, 160, 2, 2, 1)


@pytest.mark.parametrize("case", ["bad_index", "nan_vertex", "depth0", "depth13", "min_gt_depth", "bad_smoother",
                                  "bad_gpu_clip"])
def test_invalid_input_rejected_on_host(case):
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    depth, opts = 3, {}
    if case == "bad_index":
        F = F.copy(); F[1, 2] = 7
    elif case == "nan_vertex":
        V = V.copy(); V[2, 1] = np.nan
    elif case == "depth0":
        depth = 0
    elif case == "depth13":
        depth = 13
    elif case == "min_gt_depth":
        opts = {"min_depth": 5}
    elif case == "bad_smoother":
        opts = {"smoother": 9}
    elif case == "bad_gpu_clip":
        opts = {"gpu_clip": 2}
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_build_hierarchy(V, F, depth, **opts)
    assert e.value.code == 1
    if case == "bad_gpu_clip":   # the host-only build checks its options the same way, without a GPU
        with pytest.raises(L.LbmgError) as e:
            L.lbmg_host_build(V, F, depth, **opts)
        assert e.value.code == 1


def test_null_handle_rejected():
    lib = L.load_library()
    assert lib.lbmg_assemble(None, 1.0, None) == 1
    assert lib.lbmg_solve(None, None, None, 1, 1e-6, 10, 0, None, None) == 1
    assert lib.lbmg_levels(None, None, None) == 1
    assert lib.lbmg_set_area_weights(None, None, None) == 1
    assert lib.lbmg_host_levels(None, None, None) == 1
    # the learned correction and the split residual on a null handle
    assert lib.lbmg_learned_enable(None, 1, None) == 1
    assert lib.lbmg_learned_state(None, None, None, None) == 1
    assert lib.lbmg_learned_apply(None, None, 1, 1, None, None, None) == 1
    assert lib.lbmg_residual_split(None, 0, None, None, None, 1, None) == 1


def test_tune_cache_file_round_trip_and_bad_lines(tmp_path):
    """The tuning cache is plain text: valid lines load, malformed ones are reported."""
    good = tmp_path / "tune.txt"
    # eight columns, or nine with the grid of the whole-sweep kernel (threads per block 1024)
    good.write_text("# device fp64 kind lanes rows nnz threads_per_row threads_per_block [sweep_grid]\n"
                    "Test_GPU 0 0 4 1000 18000 4 128\n"
                    "Test_GPU 1 1 1 1000 18000 16 512\n"
                    "Test_GPU 0 0 4 2000 36000 4 1024 38\n")
    L.lbmg_tune_cache_load(str(good))
    out = tmp_path / "saved.txt"
    L.lbmg_tune_cache_save(str(out))
    lines = [ln.split() for ln in out.read_text().splitlines() if not ln.startswith("#")]
    assert ["Test_GPU", "0", "0", "4", "1000", "18000", "4", "128", "0"] in lines
    assert ["Test_GPU", "1", "1", "1", "1000", "18000", "16", "512", "0"] in lines
    assert ["Test_GPU", "0", "0", "4", "2000", "36000", "4", "1024", "38"] in lines
    bad = tmp_path / "bad.txt"
    # 5 threads per row is not a shape; 1024 threads per block only for a sweep with 4 per row
    bad.write_text("Test_GPU 0 0 4 1000 18000 5 128\nnot a line\nTest_GPU 0 1 4 1000 18000 4 1024 0\n")
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_tune_cache_load(str(bad))
    assert e.value.code == 1
    with pytest.raises(L.LbmgError):
        L.lbmg_tune_cache_load(str(tmp_path / "missing.txt"))


@pytest.mark.parametrize("case,code", [("no_triangles", 1), ("two_vertices", 1), ("zero_extent", 2),
                                       ("collinear", 2), ("flat_duplicate_corner", 2)])
def test_empty_and_degenerate_meshes_rejected_on_host(case, code):
    """A mesh with no triangle piece of positive area spans no basis function
    (Section 3.2 keeps only pieces of positive area): it is reported, not solved."""
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    if case == "no_triangles":
        F = np.zeros((0, 3), dtype=np.int32)
    elif case == "two_vertices":
        V, F = V[:2], np.array([[0, 1, 1]], dtype=np.int32)
    elif case == "zero_extent":
        V = np.full((4, 3), 0.25)
    elif case == "collinear":
        V = np.array([[0, 0, 0], [1, 1, 1], [2, 2, 2], [3, 3, 3]], dtype=np.float64)
    elif case == "flat_duplicate_corner":
        F = np.array([[0, 1, 1], [2, 3, 3]], dtype=np.int32)
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_build_hierarchy(V, F, 3)
    assert e.value.code == code


def test_batch_rejects_an_empty_list_and_a_bad_member():
    V = np.array([[0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]], dtype=np.float64)
    F = np.array([[0, 1, 2], [0, 1, 3]], dtype=np.int32)
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_build_batch([])
    assert e.value.code == 1
    bad = F.copy()
    bad[0, 0] = 9
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_build_batch([(V, F, 3), (V, bad, 3)])
    assert e.value.code == 1


def test_host_allocation_failure_is_reported_and_leaves_no_handle():
    """An exhausted host allocation inside the hierarchy builder (injected for the test) comes
    back as LBMG_OUT_OF_MEMORY from every build entry point, with the builder's reason, and
    the library keeps working afterwards."""
    import meshgen
    V, F = meshgen.icosphere(2)
    builds = {
        "host": lambda **o: L.lbmg_host_build(V, F, 4, **o),
        "host batch": lambda **o: L.lbmg_host_build_batch([(V, F, 4), (V, F, 3)], **o),
        "device": lambda **o: L.lbmg_build_hierarchy(V, F, 4, **o),
        "device batch": lambda **o: L.lbmg_build_batch([(V, F, 4), (V, F, 3)], **o),
    }
    for name, build in builds.items():
        with pytest.raises(L.LbmgError) as e:
            build(host_alloc_fail=1)
        assert e.value.code == 3, name
        assert "host memory exhausted" in str(e.value), name
    with pytest.raises(L.LbmgError) as e:
        L.lbmg_host_build(V, F, 4, host_alloc_fail=2)
    assert e.value.code == 1
    h = L.lbmg_host_build(V, F, 4)
    assert L.lbmg_host_levels(h)[1] == 4
    L.lbmg_host_destroy(h)
