"""Controller network kernels (forward, weighted squared error, backward,
Adam) against the FP64 reference of oracle/mlp_oracle.py, on the same BF16
weights (rounded on the host)."""
import numpy as np
import pytest

from paper_2609_19557_gb300 import mlp_data as D

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch
    assert torch.cuda.is_available()
    from paper_2609_19557_gb300 import build as B
    from paper_2609_19557_gb300 import pdnqp
    B.build()
    pdnqp.load()
    return pdnqp


def _dev(a, dtype=None):
    import torch
    t = torch.as_tensor(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def _setup(seed, batch):
    import torch
    w32 = D.init_weights(seed)
    w32[-2:] = [0.1, -0.3]
    bits = D.bf16_bits(w32)
    wq = D.bf16_values(bits).astype(np.float64)  # the weights the kernels see
    X = D.features(seed + 1, batch)
    wb = _dev(bits.view(np.int16), torch.int16)
    return w32, wq, X, wb


@pytest.mark.parametrize("batch", [1, 17, 300])
def test_forward_backward_match_oracle(P, batch):
    import torch
    from oracle import mlp_oracle as M
    w32, wq, X, wb = _setup(7, batch)
    rng = np.random.default_rng(8)
    T = rng.normal(size=(batch, 2)).astype(np.float32)
    wt = rng.uniform(0.0, 2.0, batch).astype(np.float32)
    x = _dev(X)
    y = torch.zeros((batch, 2), device="cuda")
    cache = torch.zeros((batch, 128), device="cuda")
    P.mlp_forward(wb, x, y, cache)
    Yr, cr = M.forward(wq, X.astype(np.float64))
    assert np.allclose(y.cpu().numpy(), Yr, rtol=1e-5, atol=1e-5)
    assert np.allclose(cache.cpu().numpy()[:, :64], cr["Z1"], rtol=1e-5, atol=1e-5)
    dy = torch.zeros_like(y)
    loss = torch.zeros(1, device="cuda")
    P.mlp_wmse(y, _dev(T), _dev(wt), dy, loss)
    Lr, dYr = M.wmse(Yr, T.astype(np.float64), wt.astype(np.float64))
    assert abs(loss.item() - Lr) <= 1e-5 * max(1.0, Lr)
    assert np.allclose(dy.cpu().numpy(), dYr, rtol=1e-4, atol=1e-6)
    grad = torch.zeros(P.mlp_param_count(), device="cuda")
    scratch = torch.zeros(((batch + 15) // 16) * P.mlp_param_count(), device="cuda")
    P.mlp_backward(wb, x, cache, dy, grad, scratch)
    gr = M.backward(wq, cr, dYr)
    g = grad.cpu().numpy()
    scale = np.abs(gr).max()
    assert np.abs(g - gr).max() <= 1e-4 * scale, np.abs(g - gr).max() / scale
    # deterministic: the same call gives the same bits
    grad2 = torch.zeros_like(grad)
    P.mlp_backward(wb, x, cache, dy, grad2, scratch)
    assert torch.equal(grad, grad2)


def test_adam_matches_oracle(P):
    import torch
    from oracle import mlp_oracle as M
    w32, _, _, _ = _setup(9, 1)
    rng = np.random.default_rng(10)
    g1 = rng.normal(size=w32.size).astype(np.float32)
    g2 = rng.normal(size=w32.size).astype(np.float32)
    w = _dev(w32)
    wb = torch.zeros(w32.size, dtype=torch.int16, device="cuda")
    m = torch.zeros_like(w)
    v = torch.zeros_like(w)
    th, mm, vv = w32.astype(np.float64), np.zeros(w32.size), np.zeros(w32.size)
    for step, g in ((1, g1), (2, g2)):
        P.mlp_adam(w, wb, _dev(g), m, v, step, lr=1e-2)
        th, mm, vv = M.adam_step(th, g.astype(np.float64), mm, vv, step, lr=1e-2)
    got = w.cpu().numpy().astype(np.float64)
    assert np.allclose(got, th, rtol=1e-6, atol=1e-7)
    # the BF16 copy is the nearest-even rounding of the FP32 master weights
    bits = wb.cpu().numpy().view(np.uint16)
    ref = D.bf16_bits(th.astype(np.float32))
    assert np.mean(bits == ref) > 0.999 and np.abs(bits.astype(int) - ref.astype(int)).max() <= 1


def test_training_reduces_loss(P):
    """A few hundred full-batch Adam steps with the library's kernels fit a
    smooth target."""
    import torch
    B = 512
    w32 = D.init_weights(11)
    X = D.features(12, B)
    T = np.stack([np.tanh(X[:, 0] - 0.5 * X[:, 1]), 0.3 * X[:, 2] * X[:, 3]], axis=1).astype(np.float32)
    w, x, t = _dev(w32), _dev(X), _dev(T)
    wb = torch.zeros(w32.size, dtype=torch.int16, device="cuda")
    P.mlp_to_bf16(w, wb)
    m, v = torch.zeros_like(w), torch.zeros_like(w)
    y = torch.zeros((B, 2), device="cuda")
    cache = torch.zeros((B, 128), device="cuda")
    dy, loss = torch.zeros_like(y), torch.zeros(1, device="cuda")
    grad = torch.zeros_like(w)
    scratch = torch.zeros((B // 16) * w.numel(), device="cuda")
    losses = []
    for step in range(1, 301):
        P.mlp_forward(wb, x, y, cache)
        P.mlp_wmse(y, t, None, dy, loss)
        P.mlp_backward(wb, x, cache, dy, grad, scratch)
        P.mlp_adam(w, wb, grad, m, v, step, lr=3e-3)
        if step in (1, 300):
            losses.append(loss.item())
    assert losses[1] < 0.2 * losses[0], losses
