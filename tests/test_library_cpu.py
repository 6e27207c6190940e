"""Host-side checks that need no GPU: the CUDA library builds for sm_103a,
loads, and exports every function ``include/fractal.h`` declares; the
Python binding declares the same set; the workload generators are seeded
and reproducible."""
import os
import shutil

import numpy as np
import pytest

from paper_2110_12952_gb300 import capi, workloads as W

needs_nvcc = pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                                reason="nvcc not available")


@pytest.fixture(scope="module")
def lib():
    from paper_2110_12952_gb300 import build
    if not os.path.exists(capi.LIB_PATH):
        if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
            pytest.skip("library not built and nvcc unavailable")
    build.build()
    return capi.load()


def test_header_declares_the_boundary():
    names = capi.header_functions()
    for required in ["fractal_create", "fractal_destroy", "fractal_lambda", "fractal_nu",
                     "fractal_step", "fractal_bb_step", "fractal_init_bernoulli",
                     "fractal_scatter_to_box", "fractal_gather_from_box", "fractal_last_error"]:
        assert required in names


def test_binding_covers_header():
    assert set(capi.header_functions()) <= set(capi.SIGNATURES)


@needs_nvcc
def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in capi.header_functions() if not hasattr(lib, n)]
    assert not missing
    assert b"sm_103a" in lib.fractal_version()


@needs_nvcc
def test_create_without_gpu_fails_cleanly(lib):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("GPU present")
    off = np.asarray(W.TRIANGLE.table(), dtype=np.int32).reshape(-1)
    h = capi.c_fp()
    # invalid tables are rejected before any device call
    bad = np.array([0, 0, 1, 0, 1, 0], dtype=np.int32)
    rc = lib.fractal_create(3, 2, 4, 2, bad.ctypes.data_as(capi.c_i32p), ctypes.byref(h))
    assert rc == -1 and b"duplicate" in lib.fractal_last_error()
    rc = lib.fractal_create(3, 2, 31, 2, off.ctypes.data_as(capi.c_i32p), ctypes.byref(h))
    assert rc == -2
    # a valid table needs a device: a CUDA error, not a crash
    rc = lib.fractal_create(3, 2, 4, 2, off.ctypes.data_as(capi.c_i32p), ctypes.byref(h))
    assert rc == -4 and not h.value


def test_workloads_reproducible():
    a = W.batched_mix(64, master_seed=7)
    b = W.batched_mix(64, master_seed=7)
    assert a == b
    assert {i.family.name for i in W.batched_mix(300)} == {"triangle", "carpet", "vicsek"}
    for inst in W.batched_mix(500):
        lo, hi = W.MIX_LEVELS[inst.family.name]
        assert lo <= inst.r <= hi and 0.2 <= inst.p <= 0.6 and inst.steps == 200
    tr = W.poisson_trace(duration_s=2.0)
    assert tr == W.poisson_trace(duration_s=2.0)
    t = np.array([q.arrival_s for q in tr])
    assert (np.diff(t) > 0).all() and abs(len(tr) - 4000) < 4 * np.sqrt(4000)
    assert all(10 <= q.instance.steps <= 1000 for q in tr)


def test_presets_match_their_offset_tables():
    assert W.TRIANGLE.offsets == ((0, 0), (1, 0), (0, 1))
    assert W.CARPET.k == 8 and (1, 1) not in W.CARPET.offsets
    assert W.VICSEK.offsets == ((1, 0), (0, 1), (1, 1), (2, 1), (1, 2))
    assert W.MENGER.k == 20 and W.MENGER.dim == 3
    assert W.LIFE_B3S23 == (8, 12) and W.MENGER_B5S45 == (32, 48)
