"""The allocation-free sketched-Gram entry point against the regular one (GPU).

ihsbin_sketch_gram_noalloc serves callers that cannot allocate device memory
(a host whose own pool owns all device memory, or a latency-bound caller that
cannot absorb the synchronisation of cudaMalloc/cudaFree); it keeps its split-K
partial sums in a static device array shared by all calls.  This file
is collected last so that a failure here does not hide any other test.
"""
import numpy as np
import pytest

from tests.harness import gpu_problem, small

pytestmark = pytest.mark.gpu


def _run_noalloc(lib, SA, D):
    import torch
    from paper_2210_12212_gb300 import ihsbin as ihs
    m = SA.shape[0]
    SA_dev = torch.from_numpy(np.ascontiguousarray(SA)).cuda()
    GS_dev = torch.full((D, D), float("nan"), dtype=torch.float64, device="cuda")
    st = lib.ihsbin_sketch_gram_noalloc(SA_dev.data_ptr(), m, D, GS_dev.data_ptr(), None)
    assert st == ihs.OK, lib.ihsbin_last_error()
    torch.cuda.synchronize()
    return GS_dev.cpu().numpy()


@pytest.mark.parametrize("name,kind", [("c2_small", "srht"), ("c1_small", "gaussian")])
def test_noalloc_gram_matches_regular_entry_point_twice(lib, name, kind):
    from paper_2210_12212_gb300 import ihsbin as ihs
    prob = small(name)
    ctx = ihs.Context(0)
    gp = gpu_problem(ihs, ctx, prob)
    gp.sketch(kind, prob.m, prob.s, 11)
    SA, GS = gp.sketch_matrices(prob.m, prob.d)          # the regular entry point's result
    tol = 1e-12 * np.abs(GS).max()
    for _ in range(2):                                   # two calls in a row on the shared scratch
        got = _run_noalloc(lib, SA, prob.d)
        np.testing.assert_allclose(got, GS, rtol=0, atol=tol)
    gp.close()


def test_noalloc_rejects_oversized_problem(lib):
    import torch
    from paper_2210_12212_gb300 import ihsbin as ihs
    D = 1449                                             # D*D doubles exceed the 16 MiB scratch array
    SA = torch.zeros((4, D), dtype=torch.float64, device="cuda")
    GS = torch.zeros((D, D), dtype=torch.float64, device="cuda")
    st = lib.ihsbin_sketch_gram_noalloc(SA.data_ptr(), 4, D, GS.data_ptr(), None)
    assert st == ihs.ERR_INVALID_ARG
    assert b"scratch" in lib.ihsbin_last_error()


def test_noalloc_largest_size_allocates_nothing(lib):
    """D = 1448, the largest D whose partial sums fit: the split count is cut to one, and the call
    leaves the device's free memory unchanged (measured around a second call; the first one may
    load the library's device code)."""
    import torch
    from paper_2210_12212_gb300 import ihsbin as ihs
    D, m = 1448, 8
    SA = np.random.default_rng(7).standard_normal((m, D))
    want = SA.T @ SA
    SA_dev = torch.from_numpy(SA).cuda()
    GS_dev = torch.full((D, D), float("nan"), dtype=torch.float64, device="cuda")
    for call in range(2):
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        st = lib.ihsbin_sketch_gram_noalloc(SA_dev.data_ptr(), m, D, GS_dev.data_ptr(), None)
        assert st == ihs.OK, lib.ihsbin_last_error()
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        np.testing.assert_allclose(GS_dev.cpu().numpy(), want, rtol=0, atol=1e-12 * np.abs(want).max())


def test_noalloc_rejects_huge_dimension_without_wrapping(lib):
    import torch
    from paper_2210_12212_gb300 import ihsbin as ihs
    buf = torch.zeros(16, dtype=torch.float64, device="cuda")
    st = lib.ihsbin_sketch_gram_noalloc(buf.data_ptr(), 1, 1 << 32, buf.data_ptr(), None)  # D * D wraps to 0
    assert st == ihs.ERR_INVALID_ARG
