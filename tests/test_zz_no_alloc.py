"""fractal_step_noalloc, the allocation-free variant of fractal_step, through
the C ABI.

Callers that cannot allocate device memory while they run (applications
whose device memory is handed out up front by their own pool or by another
framework, real-time loops in which cudaMalloc's possible device-wide
synchronisation is not acceptable) use this entry point; its ping-pong buffer
is a fixed device array inside the library.  Its results must equal
fractal_step's bit for bit, on consecutive calls that reuse the shared array.
This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    from paper_2110_12952_gb300 import build, capi
    build.build()
    return capi.load()


def make_handle(lib, fam, r):
    from paper_2110_12952_gb300 import capi
    off = np.ascontiguousarray(fam.table().reshape(-1))
    h = capi.c_fp()
    assert lib.fractal_create(fam.k, fam.s, r, fam.dim, off.ctypes.data_as(capi.c_i32p), ctypes.byref(h)) == 0
    levels = ctypes.c_int()
    assert lib.fractal_get_tile_levels(h, ctypes.byref(levels)) == 0   # builds the tables
    return h


def test_noalloc_matches_fractal_step_twice(lib):
    from paper_2110_12952_gb300 import workloads as W
    stream = torch.cuda.current_stream().cuda_stream
    for fam, r, rule in [(W.TRIANGLE, 11, W.LIFE_B3S23), (W.CARPET, 5, W.LIFE_B3S23),
                         (W.MENGER, 3, W.MENGER_B5S45)]:
        h = make_handle(lib, fam, r)
        cells = fam.k ** r
        for call, (seed, steps) in enumerate([(5, 7), (6, 4)]):   # two calls in a row
            x = torch.empty(cells, dtype=torch.uint8, device="cuda")
            assert lib.fractal_init_bernoulli(h, x.data_ptr(), seed, 0.4, stream) == 0
            ref = torch.empty_like(x)
            got = torch.full_like(x, 7)
            assert lib.fractal_step(h, x.data_ptr(), ref.data_ptr(), steps, rule[0], rule[1], stream) == 0
            rc = lib.fractal_step_noalloc(h, x.data_ptr(), got.data_ptr(), steps, rule[0], rule[1], stream)
            assert rc == 0, lib.fractal_last_error()
            torch.cuda.synchronize()
            assert torch.equal(got, ref), f"{fam.name} r={r} call {call}"
        assert lib.fractal_check(h) == 0
        lib.fractal_destroy(h)


def test_noalloc_allocates_nothing(lib):
    # a handle whose tables were built by fractal_get_tile_levels only (so
    # fractal_step never allocated its scratch): free device memory is the
    # same before and after a multi-generation noalloc call, and a failed
    # call's message does not outlive the next successful call
    from paper_2110_12952_gb300 import workloads as W
    stream = torch.cuda.current_stream().cuda_stream
    h = make_handle(lib, W.TRIANGLE, 12)
    x = torch.empty(3 ** 12, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    assert lib.fractal_init_bernoulli(h, x.data_ptr(), 3, 0.4, stream) == 0
    assert lib.fractal_step_noalloc(h, x.data_ptr(), y.data_ptr(), 3, 8, 12, stream) == 0
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    assert lib.fractal_step_noalloc(h, x.data_ptr(), x.data_ptr(), 3, 8, 12, stream) == -1
    assert lib.fractal_last_error() != b""
    assert lib.fractal_step_noalloc(h, x.data_ptr(), y.data_ptr(), 5, 8, 12, stream) == 0
    assert lib.fractal_last_error() == b""
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    ref = torch.empty_like(x)
    assert lib.fractal_step(h, x.data_ptr(), ref.data_ptr(), 5, 8, 12, stream) == 0
    torch.cuda.synchronize()
    assert torch.equal(y, ref)
    lib.fractal_destroy(h)


def test_noalloc_rejects_oversize_and_unprepared(lib):
    from paper_2110_12952_gb300 import capi, workloads as W
    stream = torch.cuda.current_stream().cuda_stream
    h = make_handle(lib, W.TRIANGLE, 16)          # 3^16 = 43,046,721 cells > 32 MiB
    x = torch.zeros(3 ** 16, dtype=torch.uint8, device="cuda")
    y = torch.empty_like(x)
    rc = lib.fractal_step_noalloc(h, x.data_ptr(), y.data_ptr(), 2, 8, 12, stream)
    assert rc == -1 and b"exceeds" in lib.fractal_last_error()
    lib.fractal_destroy(h)
    off = np.ascontiguousarray(W.TRIANGLE.table().reshape(-1))
    h2 = capi.c_fp()
    assert lib.fractal_create(3, 2, 6, 2, off.ctypes.data_as(capi.c_i32p), ctypes.byref(h2)) == 0
    rc = lib.fractal_step_noalloc(h2, x.data_ptr(), y.data_ptr(), 2, 8, 12, stream)
    assert rc == -1 and b"not built" in lib.fractal_last_error()
    lib.fractal_destroy(h2)
