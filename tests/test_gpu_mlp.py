"""Warm-start network kernels against the FP64 oracle (oracle/mlp.py).

Both sides round to BF16 at the same points (x, hidden activations, output and
pre-activation gradients); the kernels sum in FP32, the oracle in FP64. The
remaining differences are FP32 accumulation error (relative ~1e-6 for 256-term
sums) and the rare element whose FP32 and FP64 values straddle a BF16 rounding
boundary (one BF16 ulp, 2^-8 relative, on that element). Bars, in the max norm
relative to the largest reference entry: outputs and loss 1e-3, gradients 5e-3.
"""
import numpy as np
import pytest
import torch

from oracle import mlp as omlp
from paper_2311_01242_gb300.mlp import WarmStartMLP, init_params

pytestmark = pytest.mark.gpu

N_IN, H, N_OUT = 9, 256, 360


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _rel(a, b):
    return float(np.abs(np.asarray(a, dtype=np.float64) - b).max() / max(np.abs(b).max(), 1e-300))


def _data(seed, B):
    rng = np.random.default_rng(seed)
    x = rng.normal(size=(B, N_IN)).astype(np.float32)
    t = (0.1 * rng.normal(size=(B, N_OUT))).astype(np.float32)
    return x, t


@pytest.mark.parametrize("B", [128, 37, 1])
def test_forward_matches_oracle(B):
    p = init_params(N_IN, H, N_OUT, seed=1)
    net = WarmStartMLP(N_IN, H, N_OUT, params=p)
    x, _ = _data(2, B)
    y = net.forward(x).cpu().numpy()
    y_o, _ = omlp.forward(p.astype(np.float64), x.astype(np.float64), N_IN, H, N_OUT)
    assert y.shape == (B, N_OUT)
    assert _rel(y, y_o) <= 1e-3


@pytest.mark.parametrize("B", [128, 50])
def test_loss_and_gradient_match_oracle(B):
    p = init_params(N_IN, H, N_OUT, seed=3)
    net = WarmStartMLP(N_IN, H, N_OUT, params=p)
    x, t = _data(4, B)
    xd, td = torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda()
    loss = float(net.loss_grad(xd, td)[0])
    g = net.grads.cpu().numpy()
    loss_o, g_o = omlp.loss_grad(p.astype(np.float64), x.astype(np.float64), t.astype(np.float64), N_IN, H, N_OUT)
    assert abs(loss - loss_o) <= 1e-3 * abs(loss_o)
    lay, _ = omlp.layout(N_IN, H, N_OUT)
    for name, (o, shp) in lay.items():
        n = int(np.prod(shp))
        assert _rel(g[o:o + n], g_o[o:o + n]) <= 5e-3, name
    # padding rows/columns get exactly zero gradient
    o, shp = lay["W1"]
    assert np.all(g[o:o + shp[0] * shp[1]].reshape(shp)[:, N_IN:] == 0.0)
    o, shp = lay["W3"]
    assert np.all(g[o:o + shp[0] * shp[1]].reshape(shp)[N_OUT:, :] == 0.0)


def test_first_adam_step_closed_form():
    p = init_params(N_IN, H, N_OUT, seed=5)
    net = WarmStartMLP(N_IN, H, N_OUT, params=p)
    x, t = _data(6, 64)
    net.loss_grad(torch.as_tensor(x).cuda(), torch.as_tensor(t).cuda())
    g = net.grads.cpu().numpy().astype(np.float64)
    net.adam(lr=1e-3)
    p1 = net.params.cpu().numpy().astype(np.float64)
    want = p - 1e-3 * g / (np.abs(g) + 1e-8)
    assert np.abs(p1 - want).max() <= 1e-6
    assert int(net.step.item()) == 2


def test_training_reduces_loss_and_graph_replay_is_bitwise_eager():
    x, _ = _data(7, 96)
    t = np.tanh(x @ np.random.default_rng(8).normal(size=(N_IN, N_OUT)) * 0.3).astype(np.float32) * 0.1
    a = WarmStartMLP(N_IN, H, N_OUT, seed=9)
    b = WarmStartMLP(N_IN, H, N_OUT, seed=9)
    ha = a.fit(x, t, steps=200, lr=1e-3, use_graph=True)
    hb = b.fit(x, t, steps=200, lr=1e-3, use_graph=False)
    assert np.array_equal(ha, hb)
    assert torch.equal(a.params, b.params)
    assert ha[-1] < 0.2 * ha[0]
