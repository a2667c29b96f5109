"""Pins of the oracle's field numerics (Sec. 3.3.2, 3.4, 3.5).

  * frequency encoding: known values and the [input][k][sin, cos] order;
  * log target codec (Sec. 3.3.2, Eq. 6 and Eq. 7): exact round trip above 10^-psi and
    the clamp branch below it;
  * forward pass against a brute-force loop evaluation of a tiny network;
  * backward pass against central finite differences (FP64);
  * relative-MSE gradient against finite differences;
  * Adam's first step has the closed form w - lr g/(|g| + eps);
  * learning-rate schedule (Sec. 3.5.1) at its break points;
  * bf16 / fp16 / e4m3 rounding at ties, saturation and subnormals;
  * Kaiming-uniform init bounds and fp8 calibration scales.
"""
import math

import numpy as np
import pytest

from oracle import field as F


def test_encoding_values_and_order():
    q = np.array([[0.0, 0.5, 0.25, 1.0, 0.125, -0.5]])
    e = F.encode(q, 3).reshape(6, 3, 2)
    for d in range(6):
        for k in range(3):
            a = math.pi * (2 ** k) * q[0, d]
            assert abs(e[d, k, 0] - math.sin(a)) < 1e-15
            assert abs(e[d, k, 1] - math.cos(a)) < 1e-15
    assert e[0, 0, 0] == 0.0 and e[0, 0, 1] == 1.0
    assert abs(e[1, 0, 0] - 1.0) < 1e-15           # sin(pi/2)


def test_log_codec():
    psi = 5.0
    L = np.array([1e-4, 0.3, 1.0, 7.5, 123.0])
    Lp = F.log_encode(L, psi)
    assert np.allclose(F.log_decode(Lp, psi), L, rtol=1e-14)
    assert Lp[2] == 0.0
    assert Lp[-1] < 0.0                     # L > 1: no clamp to [0, 1]
    assert np.all(F.log_encode(np.array([0.0, 1e-6, 10.0 ** -psi]), psi) == 1.0)
    assert np.all((F.log_encode(np.array([1e-5 * 1.0001, 0.5]), psi) >= 0))


def test_forward_against_loops():
    desc = F.FieldDesc(in_freqs=1, hidden=3, n_hidden=2, prec=F.PREC_F32)
    rng = np.random.default_rng(0)
    w = rng.normal(size=desc.n_params())
    q = rng.uniform(0, 1, (4, 6))
    y, _ = F.forward(w, q, desc)
    W1 = w[:36].reshape(3, 12)
    W2 = w[36:45].reshape(3, 3)
    W3 = w[45:].reshape(3, 3)
    for b in range(4):
        feats = []
        for d in range(6):
            feats += [math.sin(math.pi * q[b, d]), math.cos(math.pi * q[b, d])]
        h1 = [max(0.0, sum(W1[o][i] * feats[i] for i in range(12))) for o in range(3)]
        h2 = [max(0.0, sum(W2[o][i] * h1[i] for i in range(3))) for o in range(3)]
        out = [sum(W3[o][i] * h2[i] for i in range(3)) for o in range(3)]
        assert np.allclose(y[b], out, rtol=1e-13, atol=1e-13)


def test_backward_finite_differences():
    desc = F.FieldDesc(in_freqs=2, hidden=8, n_hidden=3, prec=F.PREC_F32)
    rng = np.random.default_rng(1)
    w = rng.normal(size=desc.n_params()) * 0.5
    q = rng.uniform(0, 1, (16, 6))
    dy = rng.normal(size=(16, 3))
    y, cache = F.forward(w, q, desc)
    g = F.backward(w, cache, dy, desc)
    h = 1e-6
    idx = rng.choice(w.size, 60, replace=False)
    for i in idx:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (np.sum(F.forward(wp, q, desc)[0] * dy) - np.sum(F.forward(wm, q, desc)[0] * dy)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_rel_mse_gradient():
    rng = np.random.default_rng(2)
    y = rng.uniform(0, 1, (5, 3))
    yh = rng.uniform(0, 1, (5, 3))
    l, d = F.rel_mse(yh, y)
    assert abs(l - np.mean((yh - y) ** 2 / (y * y + 0.01))) < 1e-15
    h = 1e-7
    for i in range(5):
        for c in range(3):
            p, m = yh.copy(), yh.copy()
            p[i, c] += h
            m[i, c] -= h
            fd = (F.rel_mse(p, y)[0] - F.rel_mse(m, y)[0]) / (2 * h)
            assert abs(fd - d[i, c]) < 1e-7


def test_adam_first_step_closed_form():
    rng = np.random.default_rng(3)
    w = rng.normal(size=50)
    g = rng.normal(size=50)
    w1, m, v = F.adam_step(w, np.zeros(50), np.zeros(50), g, 1, 1e-2, 0.9, 0.99, 1e-8)
    assert np.allclose(w1, w - 1e-2 * g / (np.abs(g) + 1e-8), rtol=1e-13)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.01 * g * g)


def test_lr_schedule():
    # 2000 steps: decay starts at step 1400 and repeats every 25 steps
    f = lambda s: F.lr_at(s, 2000, 1e-2, 0.92, 0.7, 25)
    assert f(0) == 1e-2 and f(1399) == 1e-2
    assert abs(f(1400) - 1e-2 * 0.92) < 1e-18
    assert abs(f(1424) - 1e-2 * 0.92) < 1e-18
    assert abs(f(1425) - 1e-2 * 0.92 ** 2) < 1e-18
    assert abs(f(1999) - 1e-2 * 0.92 ** 24) < 1e-18


def test_rounding_helpers():
    one = 1.0
    assert F.round_bf16(np.array([one + 2 ** -8]))[0] == 1.0            # tie to even
    assert F.round_bf16(np.array([one + 3 * 2 ** -8]))[0] == 1.0 + 2 ** -6
    assert F.round_f16(np.array([one + 2 ** -11]))[0] == 1.0
    assert F.round_f16(np.array([one + 3 * 2 ** -11]))[0] == 1.0 + 2 ** -9
    e = F.round_e4m3(np.array([448.0, 500.0, -1e6, 2.0 ** -9, 2.0 ** -10, 1.0625, 1.1875, 0.0]))
    assert list(e) == [448.0, 448.0, -448.0, 2.0 ** -9, 0.0, 1.0, 1.25, 0.0]
    assert F.rnd(np.array([3.0]), F.PREC_FP8, 0.5)[0] == 3.0


def test_init_bounds_and_determinism():
    desc = F.FieldDesc(in_freqs=12, hidden=64, n_hidden=4, prec=F.PREC_BF16, seed=7)
    w = F.init_weights(desc)
    assert w.dtype == np.float32 and w.size == desc.n_params() == 21696
    ws = F.unflatten(w, desc)
    for W, (o, i) in zip(ws, desc.shapes()):
        b = math.sqrt(6.0 / i)
        assert np.abs(W).max() <= b
        assert abs(np.abs(W).mean() - b / 2) < 0.05 * b       # uniform on [-b, b]
    assert np.array_equal(w, F.init_weights(desc))
    assert not np.array_equal(w, F.init_weights(F.FieldDesc(12, 64, 4, F.PREC_BF16, 5.0, 8)))


def test_fp8_calibration_and_quantised_forward():
    desc = F.FieldDesc(in_freqs=12, hidden=32, n_hidden=2, prec=F.PREC_FP8, seed=1)
    w = F.init_weights(desc).astype(np.float64)
    rng = np.random.default_rng(4)
    q = rng.uniform(0, 1, (256, 6))
    s_a, s_w = F.fp8_calibrate(w, q, desc)
    assert s_a[0] == 2.0 ** -8                             # encoding amplitude 1: 1/448 -> 2^-8
    ws = F.unflatten(w, desc)
    for s, W in zip(s_w, ws[:-1]):
        a = np.abs(W).max()
        assert a / s <= 448 and a / (s / 2) > 448 and np.log2(s) == int(np.log2(s))
    assert F.pow2_scale(448.0) == 1.0 and F.pow2_scale(448.5) == 2.0
    y8, _ = F.forward(w, q, desc, (s_a, s_w))
    y32, _ = F.forward(w, q, F.FieldDesc(12, 32, 2, F.PREC_F32, 5.0, 1))
    assert np.abs(y8 - y32).max() < 0.1 * np.abs(y32).max() + 1e-3


def test_float32_encoding_of_the_tensor_core_fields(orc):
    """The kernels' float32 encoding (anchors at k = 0, 4, 8 from the own
    turn-based sine / cosine, double-angle formulas in between) against the
    exact features: within 6e-6 everywhere (three doublings of anchors good
    to 3e-7), exact at the anchors' simple arguments, negative g handled."""
    rng = np.random.default_rng(11)
    q = rng.uniform(0, 1, (20000, 6))
    q[:, 5] = rng.uniform(-0.9, 0.9, q.shape[0])
    q = np.concatenate([q, [[0, 0.25, 0.5, 0.75, 1.0, -0.5]]]).astype(np.float32).astype(np.float64)
    got = orc.encode_f32(q, 12)
    ref = F.encode(q, 12)
    assert got.shape == ref.shape
    assert np.max(np.abs(got - ref)) < 6e-6, np.max(np.abs(got - ref))
    # k = 0 features are the anchors themselves: 3e-7 (the own sine / cosine)
    k0 = np.concatenate([np.arange(24 * d, 24 * d + 2) for d in range(6)])
    assert np.max(np.abs(got[:, k0] - ref[:, k0])) < 3e-7
    # last row: v = 0 gives sin 0, cos 1 at every k
    assert np.all(got[-1, 0:24:2] == 0.0) and np.all(got[-1, 1:24:2] == 1.0)


def test_train_gradient_is_the_mean_loss_gradient():
    """Loss scaling does not change the gradient in exact arithmetic: in FP64
    without operand rounding, train_gradient equals central differences of
    the mean relative MSE (so the 1/n is applied once, not twice or never)."""
    desc = F.FieldDesc(in_freqs=2, hidden=8, n_hidden=3, prec=F.PREC_F32)
    rng = np.random.default_rng(7)
    w = rng.normal(size=desc.n_params()) * 0.5
    q = rng.uniform(0, 1, (24, 6))
    y = rng.uniform(0, 1, (24, 3))
    loss, g = F.train_gradient(w, q, y, desc)
    assert abs(loss - F.rel_mse(F.forward(w, q, desc)[0], y)[0]) < 1e-15
    h = 1e-6
    for i in rng.choice(w.size, 40, replace=False):
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (F.rel_mse(F.forward(wp, q, desc)[0], y)[0] - F.rel_mse(F.forward(wm, q, desc)[0], y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1e-3, abs(fd)), (i, fd, g[i])


def test_loss_scaled_16_bit_gradient_near_the_unrounded_one():
    """The f16 emulation's loss-scaled training gradient of a 4x128 field on
    4096 queries stays within a few % of the unrounded one (the operand
    rounding of features, activations and gradients), layer by layer."""
    desc16 = F.FieldDesc(12, 128, 4, F.PREC_F16, 5.0, 3)
    desc32 = F.FieldDesc(12, 128, 4, F.PREC_F32, 5.0, 3)
    w = F.init_weights(desc16).astype(np.float64)
    rng = np.random.default_rng(8)
    q = rng.uniform(0, 1, (4096, 6))
    q[:, 5] = rng.choice([-0.75, 0.0, 0.75], q.shape[0])
    y0, _ = F.forward(w, q, desc32)
    y = y0 + rng.normal(size=y0.shape) * 0.3          # targets near the prediction
    _, g32 = F.train_gradient(w, q, y, desc32)
    _, g16 = F.train_gradient(w, q, y, desc16)
    for a, b in zip(F.unflatten(g16, desc16), F.unflatten(g32, desc32)):
        assert np.linalg.norm(a - b) / np.linalg.norm(b) < 0.06
