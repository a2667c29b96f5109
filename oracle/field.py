"""Photon field network numerics of the oracle, in numpy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  * Input: the 6-D query (x, y, z, theta', phi', g) of Eq. 2 / Eq. 4, with the
    view direction in normalised spherical coordinates (Sec. 3.1).
  * Encoding: NeRF-style frequency encoding (Sec. 3.4 names it as the
    alternative to the hashgrid): gamma(v) = [sin(2^k pi v), cos(2^k pi v)],
    k = 0..F-1, for all six inputs, ordered [input][frequency][sin, cos].
  * Network: ReLU MLP without bias (Sec. 3.4, "no output activation"),
    Kaiming-uniform initialisation W ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)).
  * Decode: exponential decode of Eq. 7, L = 10^(-psi L').
  * Loss: relative MSE (Sec. 3.5.1), (yhat - y)^2 / (y^2 + 0.01), averaged
    over the batch and the three outputs.
  * Optimiser: Adam (Sec. 3.5.1), beta1 0.9, beta2 0.99, exponential decay of
    the learning rate by 0.92 every 25 steps from 70% of the run.

Precision emulation (how the tensor-core field is specified): the input and
the weights of every hidden layer are rounded to the field precision
(bf16 / fp16 round-to-nearest-even; fp8 e4m3 codes of x / s with per-layer
power-of-two scales s = 2^ceil(log2(amax/448)), amax taken over the weights
and over a calibration batch's layer inputs, saturating at +-448); products
are accumulated exactly
(FP64 here, FP32 on the GPU); the 3-wide output layer runs in full precision
on the unrounded last hidden activation.  In the backward pass the gradient
with respect to every hidden pre-activation is rounded to the field precision
before it is used, and the ReLU mask is taken from the rounded activation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Sequence, Tuple

import numpy as np

PREC_F32, PREC_BF16, PREC_F16, PREC_FP8 = 0, 1, 2, 3
E4M3_MAX = 448.0


@dataclasses.dataclass
class FieldDesc:
    in_freqs: int = 12
    hidden: int = 64
    n_hidden: int = 3
    prec: int = PREC_F32
    psi: float = 5.0
    seed: int = 0

    @property
    def n_in(self) -> int:
        return 12 * self.in_freqs

    def shapes(self) -> List[Tuple[int, int]]:
        s = [(self.hidden, self.n_in)]
        s += [(self.hidden, self.hidden)] * (self.n_hidden - 1)
        s += [(3, self.hidden)]
        return s

    def n_params(self) -> int:
        return sum(o * i for o, i in self.shapes())


def unflatten(flat: np.ndarray, desc: FieldDesc) -> List[np.ndarray]:
    out, o = [], 0
    for (a, b) in desc.shapes():
        out.append(np.asarray(flat[o:o + a * b], np.float64).reshape(a, b))
        o += a * b
    return out


def flatten(ws: Sequence[np.ndarray]) -> np.ndarray:
    return np.concatenate([np.asarray(w, np.float64).reshape(-1) for w in ws])


def init_weights(desc: FieldDesc) -> np.ndarray:
    """Seeded Kaiming-uniform weights as float32 master copies: element e of
    layer l draws u from Philox (tag INIT, item l, block e/4, lane e%4);
    w = (2u - 1) sqrt(6/fan_in) evaluated in FP64, then rounded once."""
    from . import philox_stream, uniform, TAG_INIT
    flat = []
    for l, (o, i) in enumerate(desc.shapes()):
        n = o * i
        nb = (n + 3) // 4
        words = philox_stream(desc.seed, TAG_INIT, 0, l + 1, nb)[l]
        u = uniform(words.reshape(-1)[:n])
        bound = math.sqrt(6.0 / i)
        flat.append(((2.0 * u - 1.0) * bound).astype(np.float32))
    return np.concatenate(flat)


# ------------------------------------------------------------------ rounding
def round_bf16(x: np.ndarray) -> np.ndarray:
    import torch
    t = torch.from_numpy(np.ascontiguousarray(x, np.float32))
    return t.to(torch.bfloat16).to(torch.float64).numpy()


def round_f16(x: np.ndarray) -> np.ndarray:
    return np.asarray(x, np.float32).astype(np.float16).astype(np.float64)


def round_e4m3(x: np.ndarray) -> np.ndarray:
    """Round to OCP fp8 e4m3 (RNE) with saturation at +-448."""
    import torch
    x = np.clip(np.asarray(x, np.float32), -E4M3_MAX, E4M3_MAX)
    t = torch.from_numpy(np.ascontiguousarray(x))
    return t.to(torch.float8_e4m3fn).to(torch.float64).numpy()


def rnd(x: np.ndarray, prec: int, scale: float = 1.0) -> np.ndarray:
    if prec == PREC_F32:
        return np.asarray(x, np.float64)
    if prec == PREC_BF16:
        return round_bf16(x)
    if prec == PREC_F16:
        return round_f16(x)
    return round_e4m3(np.asarray(x, np.float64) / scale) * scale


# ------------------------------------------------------------------ encoding / codec
def encode(q: np.ndarray, n_freq: int) -> np.ndarray:
    """gamma(v) for the six query inputs, ordered [input][k][sin, cos]."""
    q = np.asarray(q, np.float64)
    k = 2.0 ** np.arange(n_freq)
    arg = math.pi * q[:, :, None] * k[None, None, :]
    f = np.stack([np.sin(arg), np.cos(arg)], axis=-1)
    return f.reshape(q.shape[0], -1)


def log_encode(L: np.ndarray, psi: float) -> np.ndarray:
    """Target encoding (Sec. 3.3.2): -log10(L)/psi if L > 10^-psi, else 1."""
    L = np.asarray(L, np.float64)
    out = np.ones_like(L)
    m = L > 10.0 ** (-psi)
    out[m] = -np.log10(L[m]) / psi
    return out


def log_decode(Lp: np.ndarray, psi: float) -> np.ndarray:
    """Exponential decode (Eq. 7): L = 10^(-psi L')."""
    return np.power(10.0, -psi * np.asarray(Lp, np.float64))


def query_from_sample(x: np.ndarray, wo: np.ndarray, g: float) -> np.ndarray:
    """(x, theta', phi', g) with theta' = acos(w_z)/pi, phi' = atan2(w_y, w_x)/2pi mod 1."""
    x = np.asarray(x, np.float64).reshape(-1, 3)
    wo = np.asarray(wo, np.float64).reshape(-1, 3)
    th = np.arccos(np.clip(wo[:, 2], -1.0, 1.0)) / math.pi
    ph = np.arctan2(wo[:, 1], wo[:, 0]) / (2.0 * math.pi)
    ph = np.where(ph < 0.0, ph + 1.0, ph)
    return np.concatenate([x, th[:, None], ph[:, None], np.full((x.shape[0], 1), float(g))], 1)


# ------------------------------------------------------------------ network
def pow2_scale(amax: float) -> float:
    """Smallest power of two s with amax / s <= 448 (e4m3's largest finite)."""
    m, e = math.frexp(max(float(np.float32(amax)), 1e-30) / E4M3_MAX)
    return math.ldexp(1.0, e - 1 if m == 0.5 else e)


def fp8_calibrate(weights: np.ndarray, q_cal: np.ndarray, desc: FieldDesc):
    """Per-layer fp8 scales, powers of two so that x / s is exact:
    s_w from amax|W_l|, s_a from amax(layer input) over the calibration
    queries of the unquantised forward pass."""
    ws = unflatten(weights, desc)
    h = encode(q_cal, desc.in_freqs)
    s_a, s_w = [], []
    for W in ws[:-1]:
        s_a.append(pow2_scale(np.abs(h).max()))
        s_w.append(pow2_scale(np.abs(W).max()))
        h = np.maximum(h @ W.T, 0.0)
    return np.array(s_a), np.array(s_w)


def forward(weights: np.ndarray, q: np.ndarray, desc: FieldDesc, scales=None):
    """Field forward pass; returns (L' prediction (B,3), cache for backward)."""
    ws = unflatten(weights, desc)
    h = encode(q, desc.in_freqs)
    ins, zs = [], []
    L = len(ws)
    for l, W in enumerate(ws):
        if l == L - 1:
            hin, Wq = h, W
        elif desc.prec == PREC_FP8:
            s_a, s_w = scales
            hin, Wq = rnd(h, PREC_FP8, s_a[l]), rnd(W, PREC_FP8, s_w[l])
        else:
            hin, Wq = rnd(h, desc.prec), rnd(W, desc.prec)
        z = hin @ Wq.T
        ins.append(hin)
        zs.append(z)
        h = z if l == L - 1 else np.maximum(z, 0.0)
    return h, (ins, zs)


def backward(weights: np.ndarray, cache, dy: np.ndarray, desc: FieldDesc) -> np.ndarray:
    """dW = sum_b (d yhat_b / dW)^T dy_b for every layer, flattened."""
    ws = unflatten(weights, desc)
    ins, zs = cache
    L = len(ws)
    grads = [None] * L
    d = np.asarray(dy, np.float64)
    for l in range(L - 1, -1, -1):
        grads[l] = d.T @ ins[l]
        if l == 0:
            break
        Wq = ws[l] if l == L - 1 else rnd(ws[l], desc.prec)
        dh = d @ Wq
        act = np.maximum(zs[l - 1], 0.0)
        mask = rnd(act, desc.prec) > 0.0
        d = rnd(dh * mask, desc.prec)
    return flatten(grads)


def rel_mse(yhat: np.ndarray, y: np.ndarray, eps: float = 0.01):
    """Relative MSE loss and its gradient with respect to yhat."""
    diff = yhat - y
    den = y * y + eps
    n = yhat.size
    return float(np.sum(diff * diff / den) / n), 2.0 * diff / den / n


def lr_at(step: int, steps: int, lr: float, decay: float, start_frac: float, every: int) -> float:
    """Learning rate of 0-based `step`: lr * decay^k, k = number of decay
    events at steps s0, s0+every, ... <= step, s0 = ceil(start_frac*steps)."""
    s0 = int(math.ceil(start_frac * steps))
    k = 0 if step < s0 else (step - s0) // every + 1
    return lr * decay ** k


def adam_step(w, m, v, g, t: int, lr: float, b1: float, b2: float, eps: float):
    """One bias-corrected Adam update (t is 1-based); returns (w, m, v)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v
