"""FP64 oracle of the warm-start network (test infrastructure).

The learned warm start maps (r, diag h(r)) to the UCCSD angles theta at a
geometry. It is a 3-layer perceptron n_in -> H -> H -> n_out with SiLU
activations, BF16 weights and BF16 GEMM operands, whose products are summed in
higher precision. This oracle does every sum in float64 and rounds to BF16
(round to nearest, ties to even) at exactly the points where the GPU kernels
store BF16:

forward:  x_b = bf16(x); a1 = x_b W1_b^T + b1; h1_b = bf16(silu(a1));
          a2 = h1_b W2_b^T + b2; h2_b = bf16(silu(a2)); y = h2_b W3_b^T + b3
loss:     L = mean over batch and outputs of (y - t)^2
backward: dy = 2 (y - t) / (B n_out); dy_b = bf16(dy)
          dW3 = dy_b^T h2_b; db3 = sum_b dy
          da2 = (dy_b W3_b) * silu'(a2); da2_b = bf16(da2)
          dW2 = da2_b^T h1_b; db2 = sum_b da2
          da1 = (da2_b W2_b) * silu'(a1); da1_b = bf16(da1)
          dW1 = da1_b^T x_b; db1 = sum_b da1
Adam (FP32 master weights in the kernels, float64 here):
          m = b1 m + (1-b1) g; v = b2 v + (1-b2) g^2;
          w -= lr (m / (1-b1^t)) / (sqrt(v / (1-b2^t)) + eps)

Parameters are one flat array laid out as W1 [H x Ip], b1 [H], W2 [H x H],
b2 [H], W3 [Op x H], b3 [Op], with Ip = n_in rounded up to 16 and Op = n_out
rounded up to 16 (the padding columns/rows are zero).
"""
import numpy as np


def bf16_round(a):
    """Round float64/float32 values to the nearest BF16 value (ties to even),
    returned as float64. Values are first rounded to float32 (round to
    nearest even), then the float32 bit pattern is rounded to its top 16 bits."""
    f = np.asarray(a, dtype=np.float64).astype(np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def dims(n_in, n_hidden, n_out):
    ip = (n_in + 15) // 16 * 16
    op = (n_out + 15) // 16 * 16
    return ip, n_hidden, op


def layout(n_in, n_hidden, n_out):
    ip, h, op = dims(n_in, n_hidden, n_out)
    shapes = [("W1", (h, ip)), ("b1", (h,)), ("W2", (h, h)), ("b2", (h,)), ("W3", (op, h)), ("b3", (op,))]
    out, off = {}, 0
    for name, shp in shapes:
        size = int(np.prod(shp))
        out[name] = (off, shp)
        off += size
    return out, off


def unpack(params, n_in, n_hidden, n_out):
    lay, _ = layout(n_in, n_hidden, n_out)
    return {k: np.asarray(params[o:o + int(np.prod(s))], dtype=np.float64).reshape(s) for k, (o, s) in lay.items()}


def silu(a):
    return a / (1.0 + np.exp(-a))


def dsilu(a):
    s = 1.0 / (1.0 + np.exp(-a))
    return s * (1.0 + a * (1.0 - s))


def forward(params, x, n_in, n_hidden, n_out, rounding=True):
    p = unpack(params, n_in, n_hidden, n_out)
    r = bf16_round if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    ip = p["W1"].shape[1]
    xp = np.zeros((x.shape[0], ip))
    xp[:, :n_in] = x
    xb = r(xp)
    a1 = xb @ r(p["W1"]).T + p["b1"]
    h1 = r(silu(a1))
    a2 = h1 @ r(p["W2"]).T + p["b2"]
    h2 = r(silu(a2))
    y = h2 @ r(p["W3"]).T + p["b3"]
    return y[:, :n_out], dict(xb=xb, a1=a1, h1=h1, a2=a2, h2=h2, y=y, p=p)


def loss_grad(params, x, t, n_in, n_hidden, n_out, rounding=True):
    """(loss, flat gradient) with the rounding points listed in the module docstring."""
    r = bf16_round if rounding else (lambda v: np.asarray(v, dtype=np.float64))
    y, c = forward(params, x, n_in, n_hidden, n_out, rounding)
    B = x.shape[0]
    p = c["p"]
    diff = y - t
    loss = float(np.mean(diff ** 2))
    dy = np.zeros_like(c["y"])
    dy[:, :n_out] = 2.0 * diff / (B * n_out)
    dyb = r(dy)
    g = {}
    g["W3"] = dyb.T @ c["h2"]
    g["b3"] = dy.sum(axis=0)
    da2 = (dyb @ r(p["W3"])) * dsilu(c["a2"])
    da2b = r(da2)
    g["W2"] = da2b.T @ c["h1"]
    g["b2"] = da2.sum(axis=0)
    da1 = (da2b @ r(p["W2"])) * dsilu(c["a1"])
    da1b = r(da1)
    g["W1"] = da1b.T @ c["xb"]
    g["b1"] = da1.sum(axis=0)
    lay, total = layout(n_in, n_hidden, n_out)
    flat = np.zeros(total)
    for k, (o, s) in lay.items():
        flat[o:o + int(np.prod(s))] = g[k].ravel()
    # padding columns of W1 (inputs beyond n_in) carry no gradient
    o, s = lay["W1"]
    w1 = flat[o:o + s[0] * s[1]].reshape(s)
    w1[:, n_in:] = 0.0
    return loss, flat


def adam_step(params, grads, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    m = beta1 * m + (1.0 - beta1) * grads
    v = beta2 * v + (1.0 - beta2) * grads * grads
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return params - lr * mh / (np.sqrt(vh) + eps), m, v
