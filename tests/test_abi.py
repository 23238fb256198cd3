"""The C-ABI library builds, loads and exports every entry point declared in include/osvmbe.h (no GPU needed);
host-side argument checks return OSV_ERR_INVALID without touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "osvmbe.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\*?\s*(\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2106_06149_gb300 import build, osvmbe
    build.build()
    return osvmbe.load()


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ["osv_create", "osv_destroy", "clusters_build", "osv_build", "cluster_residual_solve",
              "mbe3_combine", "energy", "gradient_backward"]:
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2106_06149_gb300 import osvmbe
    names = declared_functions()
    for f in names:
        assert hasattr(lib, f), f
    assert set(names) == set(osvmbe.EXPORTS)


def test_null_and_invalid_arguments_are_rejected_on_the_host(lib):
    from paper_2106_06149_gb300 import osvmbe
    assert lib.osv_create(None, None) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_destroy(None) == osvmbe.OSV_ERR_INVALID
    assert lib.clusters_build(None, None, None, None) == osvmbe.OSV_ERR_INVALID
    assert lib.energy(None, None, None) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_syev_batched(None, 4, 1, None, None, None) == osvmbe.OSV_ERR_INVALID
    # the recorded step, the launch-shape and failure-detection settings, the counters
    assert lib.osv_graph_capture(None, None, None, 1.0, None, None) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_graph_launch(None, None, None) == osvmbe.OSV_ERR_INVALID
    n = ctypes.c_longlong()
    assert lib.osv_graph_kernels(None, ctypes.byref(n)) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_set_tridiag_variant(None, 0) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_set_wait_budget(None, 1) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_autotune(None, 1) == osvmbe.OSV_ERR_INVALID
    assert lib.osv_kernel_launches(None) == osvmbe.OSV_ERR_INVALID
