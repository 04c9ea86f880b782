"""The allocation-free Sigma^(2) entry point (for callers that cannot let the
library allocate device memory) gives what the context entry point gives.

Kept in a file of its own that pytest collects last."""
import numpy as np
import pytest

from paper_0911_4348_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
TOL = 1e-12  # the FP64 parity tolerance used throughout the GPU tests


def _maxrel(x, ref):
    return float(np.max(np.abs(x - ref)) / np.max(np.abs(ref)))


def test_noalloc_sigma2_matches_context_entry_point_on_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context, FedvrError, sigma2_noalloc
    ctx = Context()
    # two calls in a row with different shapes: the second must not see the first's leftovers
    for seed, (n, M) in enumerate([(70, 33), (37, 9)]):
        rng = W.system_rng(95, seed)
        G = torch.from_numpy(W.random_symmetric_stack(rng, M, n)).cuda()
        V = torch.from_numpy(W.random_symmetric(rng, n)).cuda()
        ref = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
        out = torch.full((M, n, n), float("nan"), dtype=torch.float64, device="cuda")
        ctx.sigma2(V, G, ref, spin=2.0)
        sigma2_noalloc(V, G, out, spin=2.0)
        torch.cuda.synchronize()
        assert _maxrel(out.cpu().numpy(), ref.cpu().numpy()) < TOL
    # sizes beyond the fixed workspace are refused, not truncated
    n, M = 200, 14
    big = torch.zeros((M, n, n), dtype=torch.float64, device="cuda")
    Vb = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    with pytest.raises(FedvrError) as e:
        sigma2_noalloc(Vb, big, big.clone())
    assert e.value.code == -1
    ctx.close()


def test_noalloc_sigma2_at_the_size_limit_allocates_nothing():
    # M n^2 = 32 * 128^2 = 2^19 is exactly the workspace limit: accepted, equal
    # to the context entry point, and a call after the first (which may load
    # the library's device code) leaves the device's free memory unchanged
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_0911_4348_gb300 import Context, FedvrError, sigma2_noalloc
    n, M = 128, 32
    rng = W.system_rng(95, 7)
    G = torch.from_numpy(W.random_symmetric_stack(rng, M, n)).cuda()
    V = torch.from_numpy(W.random_symmetric(rng, n)).cuda()
    out = torch.full((M, n, n), float("nan"), dtype=torch.float64, device="cuda")
    ref = torch.empty((M, n, n), dtype=torch.float64, device="cuda")
    sigma2_noalloc(V, G, out, spin=2.0)
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    out.fill_(float("nan"))
    sigma2_noalloc(V, G, out, spin=2.0)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    ctx = Context()
    ctx.sigma2(V, G, ref, spin=2.0)
    torch.cuda.synchronize()
    assert _maxrel(out.cpu().numpy(), ref.cpu().numpy()) < TOL
    ctx.close()
    # a negative spin factor is refused, as by the context entry point
    with pytest.raises(FedvrError) as e:
        sigma2_noalloc(V, G, out, spin=-1.0)
    assert e.value.code == -1
