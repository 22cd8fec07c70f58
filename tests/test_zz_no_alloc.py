"""ozaki_gemm_noalloc, the product entry point for callers that cannot pass a
workspace (host codes without a device allocator, or pipelines that must not
allocate mid-stream). It takes its scratch from a fixed device array inside
the library instead of a caller's buffer; it must give exactly the result of
ozaki_gemm, call after call, even though every call reuses the same array.

The file name sorts last so that a run stopping at the first failure has
already run every other test.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


def _noalloc(dmp, A, B, C, mode, s, executor):
    L = dmp.lib()
    m, k = A.shape
    n = B.shape[1]
    rc = L.ozaki_gemm_noalloc(m, n, k, A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(),
                              C.stride(0), dmp.MODES[mode], s, dmp.EXECUTORS[executor],
                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc


@pytest.mark.parametrize("executor", ["tc", "imma"])
def test_noalloc_matches_workspace_entry_point_twice(dmp, executor):
    rng = np.random.default_rng(31)
    # two calls in a row with different shapes and data: the second must not
    # see anything the first left in the shared array
    for (m, n, k, s) in [(700, 520, 900, 7), (257, 300, 129, 5)]:
        A = torch.from_numpy(rng.standard_normal((m, k)) * 0.1).cuda()
        B = torch.from_numpy(rng.standard_normal((k, n)) * 0.1).cuda()
        want = dmp.ozaki_gemm(A, B, "int8", s, executor)
        got = torch.full((m, n), float("nan"), dtype=torch.float64, device="cuda")
        assert _noalloc(dmp, A, B, got, "int8", s, executor) == dmp.OK
        assert torch.equal(got, want), (m, n, k, s)


@pytest.mark.parametrize("mode,limit", [("int8", 1056), ("e4m3", 1440)])
def test_noalloc_at_its_size_limit(dmp, mode, limit):
    """The largest square problem the header promises (s = 7, tcgen05) gives the
    bits of ozaki_gemm; one step of 32 larger is refused before any launch."""
    rng = np.random.default_rng(limit)
    A = torch.from_numpy(rng.standard_normal((limit, limit))).cuda()
    B = torch.from_numpy(rng.standard_normal((limit, limit))).cuda()
    want = dmp.ozaki_gemm(A, B, mode, 7, "tc")
    got = torch.full_like(want, float("nan"))
    assert _noalloc(dmp, A, B, got, mode, 7, "tc") == dmp.OK
    assert torch.equal(got, want)
    big = limit + 32
    Z = torch.zeros((big, big), dtype=torch.float64, device="cuda")
    C = torch.zeros_like(Z)
    before = dmp.launch_count()
    assert _noalloc(dmp, Z, Z, C, mode, 7, "tc") == dmp.ERR_WORKSPACE
    assert dmp.launch_count() == before


def test_noalloc_rejects_problems_beyond_its_array(dmp):
    A = torch.zeros((4096, 4096), dtype=torch.float64, device="cuda")
    C = torch.zeros_like(A)
    before = dmp.launch_count()
    assert _noalloc(dmp, A, A, C, "int8", 7, "tc") == dmp.ERR_WORKSPACE
    assert dmp.launch_count() == before  # rejected before any work was enqueued
