"""The allocation-free curl entry point, for callers that cannot allocate
device memory when they need the curl (it uses one static device array per
GPU instead of a context's workspaces).

Checked through the C ABI against the context-based scfft_curl (FP64), on two
calls in a row with different inputs, so a second call that reused stale
scratch from the first would fail.  This file is collected last on purpose.
"""

import ctypes

import numpy as np
import pytest

import scfft_inputs as I

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

import paper_1803_01346_gb300 as S  # noqa: E402
from paper_1803_01346_gb300 import build as B  # noqa: E402


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


def test_curl_noalloc_matches_curl_on_two_calls():
    lib = S.load_library()
    n, L = (32, 48, 16), (1.0, 1.3, 0.7)
    N = n[0] * n[1] * n[2]
    grid = S._Grid(n[0], n[1], n[2], L[0], L[1], L[2])
    stream = torch.cuda.current_stream().cuda_stream
    ctx = S.Context(n, L)
    for seed in (21, 22):
        f = torch.from_numpy(I.random_field(3 * N, seed)).cuda()
        ref = torch.empty_like(f)
        ctx.curl(f, ref)
        out = torch.full_like(f, float("nan"))
        code = lib.scfft_curl_noalloc(ctypes.byref(grid), 1.0, f.data_ptr(), out.data_ptr(),
                                      ctypes.c_void_p(stream) if stream else None)
        assert code == 0
        torch.cuda.synchronize()
        assert _rel(out, ref) < 1e-12


def test_curl_noalloc_rejects_grids_beyond_its_maximum():
    lib = S.load_library()
    grid = S._Grid(128, 128, 128, 1.0, 1.0, 1.0)
    f = torch.zeros(3 * 128 ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(f)
    assert lib.scfft_curl_noalloc(ctypes.byref(grid), 1.0, f.data_ptr(), out.data_ptr(), None) == 9


def test_curl_noalloc_near_its_maximum_on_a_side_stream():
    # 64^3 nodes fill most of the 8 MiB scratch; the call runs on a non-default stream
    lib = S.load_library()
    n, L = (64, 64, 64), (1.6, 1.6, 1.6)
    N = n[0] * n[1] * n[2]
    grid = S._Grid(n[0], n[1], n[2], L[0], L[1], L[2])
    ctx = S.Context(n, L)
    side = torch.cuda.Stream()
    for seed in (23, 24):
        f = torch.from_numpy(I.random_field(3 * N, seed)).cuda()
        ref = torch.empty_like(f)
        ctx.curl(f, ref)
        torch.cuda.synchronize()
        out = torch.full_like(f, float("nan"))
        code = lib.scfft_curl_noalloc(ctypes.byref(grid), 1.0, f.data_ptr(), out.data_ptr(),
                                      ctypes.c_void_p(side.cuda_stream))
        assert code == 0
        side.synchronize()
        assert _rel(out, ref) < 1e-12


def test_curl_noalloc_rejects_a_non_finite_sigma():
    lib = S.load_library()
    grid = S._Grid(16, 16, 16, 1.0, 1.0, 1.0)
    f = torch.zeros(3 * 16 ** 3, dtype=torch.float64, device="cuda")
    out = torch.zeros_like(f)
    assert lib.scfft_curl_noalloc(ctypes.byref(grid), float("inf"), f.data_ptr(), out.data_ptr(), None) == 1
