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


def _close(A64, x, r_ref, g_ref, r, g):
    """The product tests' tolerance: 1e-5 of the absolute sums."""
    r = np.asarray(r, np.float64)
    g = np.asarray(g, np.float64)
    ok_r = np.all(np.abs(r - r_ref) <= 1e-5 * (A64 @ np.abs(x.astype(np.float64))) + 1e-30)
    ok_g = np.all(np.abs(g - g_ref) <= 1e-5 * (A64.T @ np.abs(r_ref.astype(np.float64))) + 1e-30)
    return ok_r and ok_g


class _Problem:
    def __init__(self, tv, n, m, seed):
        self.n, self.m, self.N = n, m, n * n
        self.A = synth.gaussian_matrix(seed, m, self.N)
        self.A64 = np.abs(self.A.astype(np.float64))
        self.A_dev = torch.from_numpy(self.A).cuda()
        opt = tv.tvcs_default_options()
        opt.tau = 0.1
        self.h = tv.tvcs_create(self.A_dev, 0, m, n, 1.0, 1.0, 0.0, opt)

    def reference(self, tv, x, y):
        r_ref = np.empty(self.m, np.float32)
        g_ref = np.empty(self.N, np.float32)
        tv.tvcs_apply(self.h, x, y, r_ref, g_ref)
        return r_ref, g_ref


@pytest.mark.parametrize("n,m", [(128, 4915), (32, 307)])
def test_noalloc_matches_apply_two_calls_in_a_row(tv, n, m):
    P = _Problem(tv, n, m, 5)
    rng = np.random.default_rng(n)
    for call in range(2):
        x = rng.standard_normal(P.N).astype(np.float32)
        y = rng.standard_normal(m).astype(np.float32) if call == 0 else None
        r_ref, g_ref = P.reference(tv, x, y)
        x_dev = torch.from_numpy(x).cuda()
        y_dev = torch.from_numpy(y).cuda() if y is not None else None
        r_dev = torch.full((m,), float("nan"), dtype=torch.float32, device="cuda")
        g_dev = torch.full((P.N,), float("nan"), dtype=torch.float32, device="cuda")
        # no explicit synchronisation: the binding runs the call on torch's current
        # stream, after the copies and fills above
        tv.tvcs_apply_noalloc(P.A_dev, m, n, x_dev, y_dev, r_dev, g_dev)
        assert _close(P.A64, x, r_ref, g_ref, r_dev.cpu().numpy(), g_dev.cpu().numpy())
    tv.tvcs_destroy(P.h)


def test_noalloc_alternating_sizes_carry_nothing_over(tv):
    """Ten calls in a row alternating n = 32 and n = 128: the scratch layout changes
    between calls, and every result still equals tvcs_apply's."""
    probs = {32: _Problem(tv, 32, 307, 11), 128: _Problem(tv, 128, 4915, 12)}
    rng = np.random.default_rng(7)
    for call in range(10):
        P = probs[32 if call % 2 == 0 else 128]
        x = rng.standard_normal(P.N).astype(np.float32)
        y = rng.standard_normal(P.m).astype(np.float32)
        r_ref, g_ref = P.reference(tv, x, y)
        x_dev = torch.from_numpy(x).cuda()
        y_dev = torch.from_numpy(y).cuda()
        r_dev = torch.full((P.m,), float("nan"), dtype=torch.float32, device="cuda")
        g_dev = torch.full((P.N,), float("nan"), dtype=torch.float32, device="cuda")
        tv.tvcs_apply_noalloc(P.A_dev, P.m, P.n, x_dev, y_dev, r_dev, g_dev)
        assert _close(P.A64, x, r_ref, g_ref, r_dev.cpu().numpy(), g_dev.cpu().numpy()), call
    for P in probs.values():
        tv.tvcs_destroy(P.h)


def test_noalloc_on_a_side_stream(tv):
    """Inputs produced on a torch side stream and the call ordered on that stream."""
    P = _Problem(tv, 32, 307, 13)
    rng = np.random.default_rng(3)
    x = rng.standard_normal(P.N).astype(np.float32)
    y = rng.standard_normal(P.m).astype(np.float32)
    r_ref, g_ref = P.reference(tv, x, y)
    side = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(side):
        x_dev = torch.from_numpy(x).pin_memory().cuda(non_blocking=True)
        y_dev = torch.from_numpy(y).pin_memory().cuda(non_blocking=True)
        r_dev = torch.full((P.m,), float("nan"), dtype=torch.float32, device="cuda")
        g_dev = torch.full((P.N,), float("nan"), dtype=torch.float32, device="cuda")
        tv.tvcs_apply_noalloc(P.A_dev, P.m, P.n, x_dev, y_dev, r_dev, g_dev,
                              stream=int(side.cuda_stream))
        r_h = r_dev.cpu().numpy()
        g_h = g_dev.cpu().numpy()
    assert _close(P.A64, x, r_ref, g_ref, r_h, g_h)
    tv.tvcs_destroy(P.h)


def test_noalloc_rejects_host_pointers(tv):
    n, m = 32, 307
    N = n * n
    A_dev = torch.zeros(m * N, dtype=torch.float32, device="cuda")
    v_dev = torch.zeros(N, dtype=torch.float32, device="cuda")
    r_dev = torch.zeros(m, dtype=torch.float32, device="cuda")
    x_host = np.zeros(N, np.float32)
    r_pinned = torch.zeros(m, dtype=torch.float32).pin_memory()
    for args in [(A_dev, x_host, r_dev, v_dev), (A_dev, v_dev, r_pinned, v_dev),
                 (A_dev.cpu(), v_dev, r_dev, v_dev)]:
        with pytest.raises(tv.TvcsError) as ei:
            tv.tvcs_apply_noalloc(args[0], m, n, args[1], None, args[2], args[3])
        assert ei.value.status == tv.TVCS_ERR_INVALID_ARG and "device memory" in str(ei.value)


def test_noalloc_rejects_a_capturing_stream(tv):
    n, m = 32, 307
    N = n * n
    A_dev = torch.zeros(m * N, dtype=torch.float32, device="cuda")
    v_dev = torch.zeros(N, dtype=torch.float32, device="cuda")
    r_dev = torch.zeros(m, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    err = None
    with torch.cuda.graph(graph):
        try:
            tv.tvcs_apply_noalloc(A_dev, m, n, v_dev, None, r_dev, v_dev)
        except tv.TvcsError as e:
            err = e
        v_dev.add_(1.0)   # something for the capture to record
    assert err is not None and err.status == tv.TVCS_ERR_INVALID_ARG
    assert "capture" in str(err)
    # the device is still usable afterwards
    graph.replay()
    torch.cuda.synchronize()
    assert float(v_dev[0]) == 1.0


def test_noalloc_rejects_unsupported_sizes(tv):
    A_dev = torch.zeros(16, dtype=torch.float32, device="cuda")
    v = torch.zeros(16, dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvcsError) as ei:
        tv._check(tv._lib.tvcs_apply_noalloc(tv._ptr(A_dev), 1, 4, tv._ptr(v), None, tv._ptr(v),
                                             tv._ptr(v), None))
    assert ei.value.status == tv.TVCS_ERR_INVALID_ARG and "n = 4" in str(ei.value)
