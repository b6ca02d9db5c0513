"""The cost network's GPU kernels against the FP64 oracle: forward pass,
gradient of the mean squared error, and the Adam step; training lowers the
loss deterministically."""
import ctypes

import numpy as np
import pytest

import paper_2502_03000_gb300 as ag
from oracle import mlp as M
from tests.gpu_util import need_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    return need_gpu()


def dev(torch, a):
    return torch.tensor(np.asarray(a, dtype=np.float32), device="cuda").contiguous()


def vp(t):
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("F,H,N", [(16, 64, 1), (16, 64, 300), (5, 7, 33), (64, 128, 17)])
def test_forward_and_grad(torch, F, H, N):
    L = ag.lib()
    assert L.arma_gpu_mlp_param_count(F, H) == M.param_count(F, H)
    rng = np.random.default_rng(F * H + N)
    p = rng.normal(0, 0.3, M.param_count(F, H)).astype(np.float32)
    X = rng.normal(0, 1, (N, F)).astype(np.float32)
    T = rng.normal(0, 1, N).astype(np.float32)
    P, Xd, Td = dev(torch, p), dev(torch, X), dev(torch, T)
    y = torch.empty(N, device="cuda")
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.arma_gpu_mlp_forward(vp(P), F, H, vp(Xd), N, vp(y), st) == 0
    ref_y, _ = M.forward(p, X, F, H)
    np.testing.assert_allclose(y.cpu().numpy(), ref_y, rtol=1e-4, atol=1e-4)
    g = torch.empty(M.param_count(F, H), device="cuda")
    ws = torch.empty(int(L.arma_gpu_mlp_workspace(F, H, N)), dtype=torch.uint8, device="cuda")
    assert L.arma_gpu_mlp_grad(vp(P), F, H, vp(Xd), vp(Td), N, vp(g), None, vp(ws), ws.numel(), st) == 0
    ref_g = M.grad(p, X, T, F, H)
    got = g.cpu().numpy()
    assert np.linalg.norm(got - ref_g) <= 1e-4 * np.linalg.norm(ref_g) + 1e-7
    # deterministic: a second call gives the same bits
    g2 = torch.empty_like(g)
    assert L.arma_gpu_mlp_grad(vp(P), F, H, vp(Xd), vp(Td), N, vp(g2), None, vp(ws), ws.numel(), st) == 0
    assert torch.equal(g, g2)


def test_adam_matches_oracle(torch):
    L = ag.lib()
    rng = np.random.default_rng(5)
    n = 1000
    p, g = rng.normal(0, 1, n), rng.normal(0, 1, n)
    m, v = rng.normal(0, 0.1, n), np.abs(rng.normal(0, 0.1, n))
    P, G, Md, Vd = (dev(torch, a) for a in (p, g, m, v))
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.arma_gpu_mlp_adam(vp(P), vp(G), vp(Md), vp(Vd), n, 3, 1e-2, 0.9, 0.999, 1e-8, st) == 0
    rp, rm, rv = M.adam_step(p, g, m, v, 3, 1e-2)
    np.testing.assert_allclose(P.cpu().numpy(), rp, rtol=1e-5, atol=1e-6)
    np.testing.assert_allclose(Md.cpu().numpy(), rm, rtol=1e-5, atol=1e-7)


def test_training_fits_a_smooth_function(torch):
    """The library's kernels train the cost network: it learns a smooth
    function of its inputs (as ln(time) of the features) to well within its
    initial error."""
    from paper_2502_03000_gb300.costmodel import CostNet, HEURISTIC_FEATURE
    rng = np.random.default_rng(1)
    X = rng.normal(0, 1, (512, ag.N_FEATURES))
    T = np.sin(X[:, 0]) + 0.5 * X[:, 1] * X[:, 2] + 0.1 * X[:, 3] + X[:, HEURISTIC_FEATURE]
    net = CostNet(seed=3)
    losses = net.fit(X, T, steps=1500, lr=3e-3)
    assert losses[-1] < 0.1 * losses[0]
    pred = net.predict_log_seconds(X)
    assert np.mean((pred - T) ** 2) < 0.05
