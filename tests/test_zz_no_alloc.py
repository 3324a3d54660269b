"""ss_field_noalloc: the effective field for callers that cannot allocate device memory.

Some callers run where cudaMalloc is not theirs to call (an application that owns all device
memory through its own pool, or a plugin host that forbids allocation).  The no-allocation entry
point keeps all of its intermediates in one device array built into libss.  This file is collected
last so that a run stopping at its first failure has already run every other test.
"""
import numpy as np
import pytest
import torch

from paper_1804_07135_gb300 import workloads as W

pytestmark = pytest.mark.gpu

CASES = [
    (20, 21, 5, 1.0, 0.25, 0.1, 0.02, 3),   # ragged rows, odd image count (one pair has no partner)
    (16, 16, 1, 1.0, 0.3, 0.05, 0.01, 4),   # a different lattice on the next call: the scratch is reused
]


def _reference_field(ss, case, path32):
    with ss.StringMethod([case]) as sm:
        sm.set_path(0, path32)
        return sm.field(0, dtype=np.float32)


def test_noalloc_field_matches_ss_field_on_consecutive_calls(ss):
    for call, case in enumerate(CASES):
        nx, ny, nz, J, D, K, w, n = case
        path = W.random_spins((n, nx * ny * nz, 3), seed=40 + call).astype(np.float32)
        ref = _reference_field(ss, case, path)
        spins = torch.from_numpy(path).cuda()
        out = torch.full_like(spins, float("nan"))
        stream = torch.cuda.current_stream().cuda_stream
        ss.ss_field_noalloc(nx, ny, nz, J, D, K, w, n, spins, out, stream)
        got = out.cpu().numpy()
        assert np.isfinite(got).all()
        assert np.abs(got - ref).max() <= 1e-5 * np.abs(ref).max(), f"call {call}"


def test_noalloc_rejects_requests_beyond_its_scratch(ss):
    # 8 images of 256 x 256 x 8: the FP64 build area of the dipole spectrum alone (96*nz*Px*Py bytes,
    # about 200 MB) exceeds the built-in 32 MiB array, so the call returns before touching the GPU.
    dummy = torch.zeros(16, device="cuda")
    p = dummy.data_ptr()
    import ctypes
    st = ss._lib.ss_field_noalloc(256, 256, 8, 1.0, 0.3, 0.05, 0.01, 8, ctypes.c_void_p(p), ctypes.c_void_p(p), None)
    assert st == ss.SS_ERR_INVALID_ARG
    assert torch.count_nonzero(dummy).item() == 0
