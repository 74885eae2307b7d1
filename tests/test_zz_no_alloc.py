"""The allocation-free 2D Euler right-hand side (enomr_rhs_euler2d_noalloc).

It serves callers that cannot call cudaMalloc -- a host framework that owns
the device memory through its own caching allocator, a program with a fixed
memory budget, or a latency-sensitive loop in which cudaMalloc/cudaFree
would synchronise the device.  Its scratch is a static device array shared
by every call.  The test calls it through the C ABI twice in a row (the
second call sees the first call's leftovers in that array) and checks both
results against enomr_rhs of a context with the same parameters, within the
value tolerance of the parity tests.  This file is collected last so that a
run stopping at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

from paper_2311_15504_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


def test_noalloc_rhs_matches_context_rhs():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as ge
    ge.build_cuda()
    from paper_2311_15504_gb300 import enomr

    lib = enomr._lib
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    cases = [  # two different problems back to back, then the first again
        (9, 1, wl.riemann2d(300, 140, seed=11)),
        (13, 0, (wl.smooth_random_euler2d(133, 70, seed=3), 1.0 / 133, 1.0 / 70)),
        (9, 1, wl.riemann2d(300, 140, seed=11)),
    ]
    for order, bc, (U, dx, dy) in cases:
        ny, nx = U.shape[1], U.shape[2]
        Ud = torch.from_numpy(U).cuda()
        ref = enomr.Solver(enomr.EULER, (ny, nx), order=order, dx=dx, dy=dy, bc=bc).rhs(Ud)
        for _ in range(2):
            out = torch.full_like(Ud, float("nan"))
            st = lib.enomr_rhs_euler2d_noalloc(ctypes.c_void_p(Ud.data_ptr()),
                                               ctypes.c_void_p(out.data_ptr()), nx, ny, dx, dy,
                                               order, 1.4, bc, stream)
            assert st == 0, lib.enomr_strerror(st)
            torch.cuda.synchronize()
            scale = max(float(ref.abs().max()), 1e-300)
            err = float((out - ref).abs().max()) / scale
            assert err <= 1e-12, err

    # sizes beyond the static scratch are rejected before any launch
    big = 16385
    st = lib.enomr_rhs_euler2d_noalloc(ctypes.c_void_p(1), ctypes.c_void_p(2), big, 8, 0.1, 0.1,
                                       9, 1.4, 1, stream)
    assert st == 1
