"""tvcs_apply_noalloc -- the products entry point that allocates no device
memory, for callers that cannot call cudaMalloc when they need the products
(device memory fully reserved by their own pool, a hard memory cap, or loops
that cannot afford an allocation's implicit synchronisation).  Its results
must match the regular tvcs_apply on the same data, call after call, although
every call reuses one file-scope scratch array."""
import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tv(cuda_device):
    import __graft_entry__
    __graft_entry__.build()
    import paper_1001_1774_gb300 as tv
    return tv


@pytest.mark.parametrize("n,m", [(128, 4915), (32, 307)])
def test_noalloc_matches_apply_two_calls_in_a_row(tv, n, m):
    N = n * n
    A = synth.gaussian_matrix(5, m, N)
    A64 = np.abs(A.astype(np.float64))
    A_dev = torch.from_numpy(A).cuda()
    opt = tv.tvcs_default_options()
    opt.tau = 0.1
    h = tv.tvcs_create(A_dev, 0, m, n, 1.0, 1.0, 0.0, opt)
    rng = np.random.default_rng(n)
    for call in range(2):
        x = rng.standard_normal(N).astype(np.float32)
        y = rng.standard_normal(m).astype(np.float32) if call == 0 else None
        r_ref = np.empty(m, np.float32)
        g_ref = np.empty(N, np.float32)
        tv.tvcs_apply(h, x, y, r_ref, g_ref)
        x_dev = torch.from_numpy(x).cuda()
        y_dev = torch.from_numpy(y).cuda() if y is not None else None
        r_dev = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
        g_dev = torch.full((N,), float("nan"), dtype=torch.float32, device="cuda")
        torch.cuda.synchronize()
        tv.tvcs_apply_noalloc(A_dev, m, n, x_dev, y_dev, r_dev, g_dev)
        r = r_dev.cpu().numpy().astype(np.float64)
        g = g_dev.cpu().numpy().astype(np.float64)
        # the product tests' tolerance: 1e-5 of the absolute sums
        assert np.all(np.abs(r - r_ref) <= 1e-5 * (A64 @ np.abs(x.astype(np.float64))) + 1e-30)
        assert np.all(np.abs(g - g_ref) <= 1e-5 * (A64.T @ np.abs(r_ref.astype(np.float64))) + 1e-30)
    tv.tvcs_destroy(h)


def test_noalloc_rejects_unsupported_sizes(tv):
    A_dev = torch.zeros(16, dtype=torch.float32, device="cuda")
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvcsError) as ei:
        tv._check(tv._lib.tvcs_apply_noalloc(tv._ptr(A_dev), 1, 4, tv._ptr(v), None, tv._ptr(v),
                                             tv._ptr(v), None))
    assert ei.value.status == tv.TVCS_ERR_INVALID_ARG and "n = 4" in str(ei.value)
