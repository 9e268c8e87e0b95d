"""The allocation-free residual norm, rgs_residual_norm_noalloc, against rgs_solve's own norms.

This entry point exists for callers that cannot allocate device memory themselves: a host
application that has already reserved its whole device budget and only lends the library
buffers it owns, or a latency-critical loop that cannot afford the device-wide
synchronisation of cudaMalloc.  Its scratch lives in a static device array inside the
library.  The test calls it through the C ABI twice in a row, on consecutive pairs of
iterates of a real solve, and requires both results to match the FP64 per-bounce norms
that rgs_solve reports, within the tolerance of the other GPU tests.  The file is named to
be collected last, so that a run stopping at its first failure has run everything else.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-4  # the relative tolerance of the FP32 GPU tests


def test_noalloc_residual_norm_matches_solve_norms():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import api, build, rgs, scenes

    build.build()
    L = rgs.load()
    sc = scenes.box_scene(n=1200, nd=64, nb=3)
    d = api.upload(sc)
    pipe = api.Pipeline()
    pipe.build(d)
    pipe.trace(d)
    _, stats = pipe.solve(None, 3, stats=True)
    iters = [rgs.rgs_get_iterate(pipe.transport, b) for b in range(4)]
    torch.cuda.synchronize()

    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    n = iters[0].numel()
    for call, b in enumerate((1, 2)):  # two calls in a row, sharing the static scratch
        st = L.rgs_residual_norm_noalloc(ct.c_void_p(iters[b].data_ptr()), ct.c_void_p(iters[b - 1].data_ptr()),
                                         ct.c_int64(n), ct.c_void_p(out[call].data_ptr()), stream)
        assert st == 0, L.rgs_last_error()
    torch.cuda.synchronize()
    got = out.cpu().numpy()
    want = np.array(stats["residual_norm"][:2])
    assert np.all(want > 0) and got[0] != got[1]
    np.testing.assert_allclose(got, want, rtol=TOL)

    # sizes beyond the fixed scratch are refused on the host, with a message
    st = L.rgs_residual_norm_noalloc(ct.c_void_p(iters[1].data_ptr()), ct.c_void_p(iters[0].data_ptr()),
                                     ct.c_int64(8192 * 8192 + 1), ct.c_void_p(out[0].data_ptr()), stream)
    assert st == 1 and b"outside" in L.rgs_last_error()


def test_noalloc_residual_norm_empty_and_full_scratch():
    """n = 0 launches no partial block and still writes 0; n at the limit fills all 8,192
    scratch slots (x = y gives exactly 0; a one-element difference in the last slot's block
    gives exactly its magnitude, so that slot was summed too)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2509_18497_gb300 import build, rgs

    build.build()
    L = rgs.load()
    stream = ct.c_void_p(torch.cuda.current_stream().cuda_stream)
    out = torch.full((3,), -1.0, dtype=torch.float64, device="cuda")
    x = torch.zeros(8192 * 8192, dtype=torch.float32, device="cuda")
    y = x.clone()
    y[-1] = 0.75
    for call, (n, a, b) in enumerate(((0, x, y), (x.numel(), x, x), (x.numel(), x, y))):
        st = L.rgs_residual_norm_noalloc(ct.c_void_p(a.data_ptr()), ct.c_void_p(b.data_ptr()), ct.c_int64(n),
                                         ct.c_void_p(out[call].data_ptr()), stream)
        assert st == 0, L.rgs_last_error()
    torch.cuda.synchronize()
    assert out.cpu().tolist() == [0.0, 0.0, 0.75]
    # the binding checks devices and runs on x's device
    got = rgs.rgs_residual_norm_noalloc(x[:1000], y[:1000])
    assert float(got) == 0.0
