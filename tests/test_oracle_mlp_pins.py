"""Pins of the warm-start network oracle (oracle/mlp.py)."""
import numpy as np

from oracle import mlp


def test_bf16_rounding_is_round_to_nearest_even():
    # BF16 keeps the top 16 bits of an FP32 value: 8 significand bits.
    one = 1.0
    ulp = 2.0 ** -7  # spacing of BF16 values in [1, 2)
    cases = [
        (one, one),
        (one + ulp, one + ulp),                   # representable
        (one + ulp / 2, one),                     # tie, 1.0 has an even significand
        (one + 3 * ulp / 2, one + 2 * ulp),       # tie, rounds to the even neighbour
        (one + ulp / 2 + 2.0 ** -20, one + ulp),  # just above the tie
        (one + ulp / 2 - 2.0 ** -20, one),        # just below the tie
        (-(one + 3 * ulp / 2), -(one + 2 * ulp)),
        (0.0, 0.0),
        (2.0 ** -130, 2.0 ** -130),               # FP32 subnormal with few bits stays exact
    ]
    for a, want in cases:
        assert mlp.bf16_round(np.array([a]))[0] == want, a
    # every output is a BF16 value: low 16 bits of its FP32 pattern are zero
    r = mlp.bf16_round(np.random.default_rng(0).normal(size=1000))
    assert np.all((r.astype(np.float32).view(np.uint32) & 0xFFFF) == 0)


def test_layout_and_padding():
    lay, total = mlp.layout(9, 256, 360)
    assert lay["W1"][1] == (256, 16) and lay["W3"][1] == (368, 256)
    assert total == 256 * 16 + 256 + 256 * 256 + 256 + 368 * 256 + 368
    lay, total = mlp.layout(3, 16, 5)
    assert lay["W3"][1] == (16, 16) and lay["b3"][1] == (16,)


def _tiny(seed=0, n_in=3, h=16, n_out=5, B=7):
    rng = np.random.default_rng(seed)
    lay, total = mlp.layout(n_in, h, n_out)
    p = rng.normal(0, 0.4, size=total)
    o, s = lay["W1"]
    w1 = p[o:o + s[0] * s[1]].reshape(s)
    w1[:, n_in:] = 0.0
    o, s = lay["W3"]
    w3 = p[o:o + s[0] * s[1]].reshape(s)
    w3[n_out:, :] = 0.0
    o, s = lay["b3"]
    p[o + n_out:o + s[0]] = 0.0
    x = rng.normal(size=(B, n_in))
    t = rng.normal(size=(B, n_out))
    return p, x, t, (n_in, h, n_out)


def test_unrounded_gradient_matches_finite_differences():
    p, x, t, d = _tiny()
    loss, g = mlp.loss_grad(p, x, t, *d, rounding=False)
    rng = np.random.default_rng(1)
    lay, total = mlp.layout(*d)
    live = [i for i in range(total) if abs(g[i]) > 0 or rng.random() < 0.05]
    idx = rng.choice(live, size=40, replace=False)
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        fd = (mlp.loss_grad(pp, x, t, *d, rounding=False)[0] - mlp.loss_grad(pm, x, t, *d, rounding=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-8 + 1e-6 * abs(fd), (i, fd, g[i])


def test_silu_derivative_closed_form():
    a = np.linspace(-6, 6, 101)
    h = 1e-6
    fd = (mlp.silu(a + h) - mlp.silu(a - h)) / (2 * h)
    assert np.abs(fd - mlp.dsilu(a)).max() < 1e-8
    assert abs(mlp.silu(0.0)) == 0.0 and abs(mlp.dsilu(0.0) - 0.5) < 1e-15


def test_rounded_forward_is_near_unrounded():
    p, x, t, d = _tiny(3)
    y_r, _ = mlp.forward(p, x, *d, rounding=True)
    y_u, _ = mlp.forward(p, x, *d, rounding=False)
    # BF16 carries 8 significand bits: relative perturbations of order 2^-8 per stage
    assert np.abs(y_r - y_u).max() <= 0.05 * np.abs(y_u).max()
    assert not np.array_equal(y_r, y_u)


def test_first_adam_step_is_signed_learning_rate():
    """With zero moments, step 1 gives m_hat = g and v_hat = g^2, so every weight
    with a nonzero gradient moves by lr * g / (|g| + eps)."""
    rng = np.random.default_rng(4)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    g[:5] = 0.0
    w1, m, v = mlp.adam_step(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.allclose(w1 - w, -1e-3 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=1e-15)
    assert np.array_equal(w1[:5], w[:5])
