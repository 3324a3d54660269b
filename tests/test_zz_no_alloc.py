"""ss_field_noalloc: the effective field for callers that cannot allocate device memory.

Some callers run where cudaMalloc is not theirs to call (an application that owns all device
memory through its own pool, or a plugin host that forbids allocation).  The no-allocation entry
point keeps all of its intermediates in one device array built into libss.  Each case is compared
with the FP64 oracle's field (Eqs. 2-7) and with ss_field of an FP32 context, within the FP32 field
tolerance the other parity tests use (1e-5 of max |h|), on consecutive calls that reuse the array.
This file is collected last so that a run stopping at its first failure has already run every other
test.
"""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    (20, 21, 5, 1.0, 0.25, 0.1, 0.02, 3),   # ragged rows, odd image count (one pair has no partner)
    (16, 16, 1, 1.0, 0.3, 0.05, 0.01, 4),   # a different lattice on the next call: the scratch is reused
    (64, 64, 4, 1.0, 0.25, 0.1, 0.02, 2),   # padded length 128: the two-pass x and y/z kernels
    (12, 10, 3, 1.0, 0.3, 0.05, 0.0, 3),    # w = 0: no dipole term, no spectrum (Px = Py = 1)
]


def _unit(a):
    return a / np.linalg.norm(a, axis=-1, keepdims=True)


def _ss_field(ss, case, path32):
    with ss.StringMethod([case]) as sm:
        sm.set_path(0, path32)
        return sm.field(0, dtype=np.float32)


def test_noalloc_field_matches_the_oracle_on_consecutive_calls(ss):
    stream = torch.cuda.current_stream().cuda_stream
    for call, case in enumerate(CASES):
        nx, ny, nz, J, D, K, w, n = case
        path = W.random_spins((n, nx * ny * nz, 3), seed=40 + call).astype(np.float32)
        spins = torch.from_numpy(path).cuda()
        out = torch.full_like(spins, float("nan"))
        ss.ss_field_noalloc(nx, ny, nz, J, D, K, w, n, spins, out, stream)
        got = out.cpu().numpy()
        assert np.isfinite(got).all(), f"call {call}"
        ref = oracle.field(oracle.model(nx, ny, nz, J, D, K, w), _unit(path.astype(np.float64)))
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), f"call {call}: against the oracle"
        ctx = _ss_field(ss, case, path)
        assert np.abs(got - ctx).max() <= 1e-5 * np.abs(ref).max(), f"call {call}: against ss_field"


def test_noalloc_rejects_requests_beyond_its_scratch(ss):
    # 8 images of 256 x 256 x 8: the FP64 build area of the dipole spectrum alone (96*nz*Px*Py bytes,
    # about 200 MB) exceeds the built-in 32 MiB array, so the call returns before touching the GPU.
    dummy = torch.zeros(16, device="cuda")
    p = dummy.data_ptr()
    st = ss._lib.ss_field_noalloc(256, 256, 8, 1.0, 0.3, 0.05, 0.01, 8, ctypes.c_void_p(p), ctypes.c_void_p(p), None)
    assert st == ss.SS_ERR_INVALID_ARG
    assert torch.count_nonzero(dummy).item() == 0


def test_noalloc_rejects_memory_that_is_not_on_the_device(ss):
    # The pointer check runs on the host before any launch.  Page-locked host buffers are used: they
    # are reachable from the GPU, so even a missing check could not fault it.
    nx, ny, nz, n = 8, 8, 1, 2
    host_in = torch.ones((n, nx * ny * nz, 3), dtype=torch.float32).pin_memory()
    host_out = torch.zeros_like(host_in).pin_memory()
    dev = torch.ones((n, nx * ny * nz, 3), dtype=torch.float32, device="cuda")
    f = ss._lib.ss_field_noalloc
    for a, b in ((host_in, dev), (dev, host_out)):
        st = f(nx, ny, nz, 1.0, 0.3, 0.05, 0.01, n, ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()), None)
        assert st == ss.SS_ERR_INVALID_ARG
    assert torch.count_nonzero(host_out).item() == 0


def test_noalloc_refuses_a_capturing_stream(ss):
    nx, ny, nz, n = 8, 8, 1, 2
    spins = torch.ones((n, nx * ny * nz, 3), dtype=torch.float32, device="cuda")
    out = torch.zeros_like(spins)
    s = torch.cuda.Stream()
    g = torch.cuda.CUDAGraph()
    status = {}
    with torch.cuda.graph(g, stream=s):
        status["st"] = ss._lib.ss_field_noalloc(nx, ny, nz, 1.0, 0.3, 0.05, 0.01, n, ctypes.c_void_p(spins.data_ptr()),
                                                ctypes.c_void_p(out.data_ptr()), ctypes.c_void_p(s.cuda_stream))
        out.add_(0.0)  # the capture still records torch's own work
    assert status["st"] == ss.SS_ERR_STATE
    g.replay()
    torch.cuda.synchronize()
    assert torch.count_nonzero(out).item() == 0
