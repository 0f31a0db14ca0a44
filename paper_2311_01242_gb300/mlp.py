"""The warm-start network on the GPU (binding of the vqe_mlp_* entry points).

A 3-layer perceptron with BF16 weights on the tensor cores and FP32
accumulation, trained by Adam on FP32 master weights; all arithmetic runs in
libvqe's kernels, torch only holds the buffers. One training step (loss and
gradient, then the Adam update) can be captured once in a CUDA graph and
replayed, since the Adam step counter lives on the device.
"""
import ctypes

import numpy as np
import torch

from . import _native
from .api import _check, _ptr, _stream


def param_layout(n_in, n_hidden, n_out):
    """Offsets and shapes of W1, b1, W2, b2, W3, b3 in the flat parameter array."""
    ip = (n_in + 15) // 16 * 16
    op = (n_out + 15) // 16 * 16
    shapes = [("W1", (n_hidden, ip)), ("b1", (n_hidden,)), ("W2", (n_hidden, n_hidden)), ("b2", (n_hidden,)),
              ("W3", (op, n_hidden)), ("b3", (op,))]
    out, off = {}, 0
    for name, shp in shapes:
        out[name] = (off, shp)
        off += int(np.prod(shp))
    return out, off


def init_params(n_in, n_hidden, n_out, seed=0):
    """Uniform(-1/sqrt(fan_in), 1/sqrt(fan_in)) weights and biases; padding zero."""
    rng = np.random.default_rng(seed)
    lay, total = param_layout(n_in, n_hidden, n_out)
    p = np.zeros(total, dtype=np.float32)
    fans = {"W1": n_in, "b1": n_in, "W2": n_hidden, "b2": n_hidden, "W3": n_hidden, "b3": n_hidden}
    for name, (o, shp) in lay.items():
        bound = 1.0 / np.sqrt(fans[name])
        vals = rng.uniform(-bound, bound, size=shp).astype(np.float32)
        if name == "W1":
            vals[:, n_in:] = 0.0
        if name == "W3":
            vals[n_out:, :] = 0.0
        if name == "b3":
            vals[n_out:] = 0.0
        p[o:o + vals.size] = vals.ravel()
    return p


class WarmStartMLP:
    def __init__(self, n_in, n_hidden, n_out, seed=0, device="cuda", params=None):
        self.lib = _native.load()
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        n = int(self.lib.vqe_mlp_param_count(self.n_in, self.n_hidden, self.n_out))
        if n <= 0:
            raise ValueError(self.lib.vqe_last_error().decode())
        p = init_params(n_in, n_hidden, n_out, seed) if params is None else np.asarray(params, dtype=np.float32)
        assert p.size == n
        self.device = torch.device(device)
        self.params = torch.as_tensor(p).to(self.device).contiguous()
        self.params_bf16 = torch.empty(n, dtype=torch.int16, device=self.device)
        self.grads = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.m = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.v = torch.zeros(n, dtype=torch.float32, device=self.device)
        self.step = torch.ones(1, dtype=torch.int32, device=self.device)
        self.loss = torch.zeros(1, dtype=torch.float32, device=self.device)
        self.n_params = n
        self._ws = {}
        self._graph = None
        _check(self.lib.vqe_mlp_to_bf16(n, _ptr(self.params), _ptr(self.params_bf16), _stream()))

    def _workspace(self, batch):
        if batch not in self._ws:
            nb = int(self.lib.vqe_mlp_workspace_bytes(batch, self.n_in, self.n_hidden, self.n_out))
            self._ws[batch] = torch.empty(nb, dtype=torch.uint8, device=self.device)
        return self._ws[batch]

    def forward(self, x, y=None):
        x = torch.as_tensor(x, dtype=torch.float32).to(self.device).contiguous()
        B = x.shape[0]
        if y is None:
            y = torch.empty(B, self.n_out, dtype=torch.float32, device=self.device)
        ws = self._workspace(B)
        _check(self.lib.vqe_mlp_forward(B, self.n_in, self.n_hidden, self.n_out, _ptr(x), _ptr(self.params),
                                        _ptr(self.params_bf16), _ptr(y), _ptr(ws), ws.numel(), _stream()))
        return y

    def loss_grad(self, x, t):
        """Loss (device scalar) and gradient (into self.grads) for a batch."""
        B = x.shape[0]
        ws = self._workspace(B)
        _check(self.lib.vqe_mlp_loss_grad(B, self.n_in, self.n_hidden, self.n_out, _ptr(x), _ptr(t),
                                          _ptr(self.params), _ptr(self.params_bf16), _ptr(self.grads),
                                          _ptr(self.loss), _ptr(ws), ws.numel(), _stream()))
        return self.loss

    def adam(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        _check(self.lib.vqe_mlp_adam(self.n_params, _ptr(self.params), _ptr(self.grads), _ptr(self.m),
                                     _ptr(self.v), _ptr(self.step), float(lr), float(beta1), float(beta2),
                                     float(eps), _ptr(self.params_bf16), _stream()))

    def train_step(self, x, t, lr=1e-3):
        self.loss_grad(x, t)
        self.adam(lr)
        return self.loss

    def fit(self, x, t, steps, lr=1e-3, use_graph=True):
        """Full-batch Adam for `steps` steps; returns the loss history (host)."""
        x = torch.as_tensor(x, dtype=torch.float32).to(self.device).contiguous()
        t = torch.as_tensor(t, dtype=torch.float32).to(self.device).contiguous()
        hist = torch.empty(steps, dtype=torch.float32, device=self.device)
        if not use_graph:
            for i in range(steps):
                self.train_step(x, t, lr)
                hist[i] = self.loss[0]
            return hist.cpu().numpy()
        # warm up once outside capture (workspace allocation), then capture one step
        self._workspace(x.shape[0])
        self.train_step(x, t, lr)
        hist[0] = self.loss[0]
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream())
        g = torch.cuda.CUDAGraph()
        with torch.cuda.stream(side):
            with torch.cuda.graph(g, stream=side):
                self.train_step(x, t, lr)
        torch.cuda.current_stream().wait_stream(side)
        for i in range(1, steps):
            g.replay()
            hist[i] = self.loss[0]
        self._graph = g
        return hist.cpu().numpy()
