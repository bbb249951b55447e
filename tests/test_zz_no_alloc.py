"""pdnqp_kkt_residuals_noalloc: the allocation-free variant of the external
KKT test, for callers that cannot call cudaMalloc / cudaFree (for example a
runtime whose memory manager owns all device memory, or a latency-critical
loop that cannot afford cudaFree's device-wide synchronisation).  Its scratch
is a static device array shared by all calls, so the test calls it twice in a
row with different points and compares each result with the allocating entry
point, through the C ABI.  Collected last so that a failure here does not stop
the other tests of a run that stops at the first failure."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import instances as I

pytestmark = pytest.mark.gpu


def test_noalloc_matches_allocating_entry_point():
    import torch
    from paper_2609_19557_gb300 import build as B
    from paper_2609_19557_gb300 import pdnqp as P
    assert torch.cuda.is_available()
    B.build()
    P.load()
    inst = I.mid_qp(2)  # n = 50,000: many blocks per pass
    prob = P.DeviceProblem(inst)
    n, m = prob.n, prob.m
    rng = np.random.default_rng(11)
    stream = torch.cuda.current_stream()
    for call in range(2):
        x = torch.as_tensor(np.clip(rng.normal(scale=0.5 + call, size=n), -3, 3), device="cuda")
        y = torch.as_tensor(rng.normal(scale=1 + 5 * call, size=m), device="cuda")
        ref = torch.zeros(4, device="cuda", dtype=torch.float64)
        P.pdnqp_kkt_residuals(prob, x, y, ref, stream=stream.cuda_stream)
        got = torch.full((4,), float("nan"), device="cuda", dtype=torch.float64)
        P.pdnqp_kkt_residuals_noalloc(prob, x, y, got, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.all(np.isfinite(g)), g
        assert np.allclose(g, r, rtol=1e-12, atol=1e-14), (call, g, r)
