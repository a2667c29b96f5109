"""Photon field network numerics of the oracle, in numpy FP64.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

  * Input: the 6-D query (x, y, z, theta', phi', g) of Eq. 2 / Eq. 4, with the
    view direction in normalised spherical coordinates (Sec. 3.1).
  * Encoding: NeRF-style frequency encoding (Sec. 3.4 names it as the
    alternative to the hashgrid): gamma(v) = [sin(2^k pi v), cos(2^k pi v)],
    k = 0..F-1, for all six inputs, ordered [input][frequency][sin, cos];
    or the paper's own multiresolution hash-grid encoding (Sec. 3.4, after
    Mueller et al. 2022), one 3-D grid for the position and one 2-D grid for
    the direction, g passed through raw (see hash_encode).
  * Network: ReLU MLP without bias (Sec. 3.4, "no output activation"),
    Kaiming-uniform initialisation W ~ U(-sqrt(6/fan_in), sqrt(6/fan_in)).
  * Decode: exponential decode of Eq. 7, L = 10^(-psi L').
  * Loss: relative MSE (Sec. 3.5.1), (yhat - y)^2 / (y^2 + 0.01), averaged
    over the batch and the three outputs.
  * Optimiser: Adam (Sec. 3.5.1), beta1 0.9, beta2 0.99, exponential decay of
    the learning rate by 0.92 every 25 steps from 70% of the run.

Precision emulation (how the tensor-core field is specified): the encoding
is taken in the float32 steps of the kernels (encode_f32: own turn-based
sine / cosine at every fourth frequency, double-angle formulas in between,
within a few 1e-6 of the exact features); the input and the weights of every
hidden layer are rounded to the field precision
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
ENC_FREQUENCY, ENC_HASHGRID = 0, 1
E4M3_MAX = 448.0
HASH_PRIMES = (1, 2654435761, 805459861)
HASH_INIT = 1e-4


@dataclasses.dataclass
class HashGrid:
    """One multiresolution hash grid over [0,1]^dim: level l has resolution
    N_l = floor(base_res * scale^l) cells per axis, (N_l + 1)^dim vertices,
    and a table of min((N_l + 1)^dim, 2^log2_size) entries of `features`
    floats; a level whose vertices fit is indexed densely (x fastest), the
    others by the spatial hash (xor of v_k * pi_k, pi = 1, 2654435761,
    805459861, in 32-bit arithmetic) modulo the table size."""
    dim: int
    levels: int
    features: int
    log2_size: int
    base_res: int
    scale: float

    def res(self, l: int) -> int:
        # scale^l by repeated FP64 products of the float32 scale, as the library does
        s = 1.0
        for _ in range(l):
            s *= float(np.float32(self.scale))
        return int(math.floor(self.base_res * s))

    def dense(self, l: int) -> bool:
        return (self.res(l) + 1) ** self.dim <= 2 ** self.log2_size

    def entries(self, l: int) -> int:
        return (self.res(l) + 1) ** self.dim if self.dense(l) else 2 ** self.log2_size

    def level_floats(self, l: int) -> int:
        # tables start on 8-float boundaries
        return (self.entries(l) * self.features + 7) // 8 * 8

    def n_params(self) -> int:
        return sum(self.level_floats(l) for l in range(self.levels))


@dataclasses.dataclass
class FieldDesc:
    in_freqs: int = 12
    hidden: int = 64
    n_hidden: int = 3
    prec: int = PREC_F32
    psi: float = 5.0
    seed: int = 0
    encoding: int = ENC_FREQUENCY
    hash_levels: int = 16
    hash_features: int = 8
    hash_log2_size: int = 19
    hash_base_res: int = 16
    hash_scale: float = 2.0

    def grids(self) -> List[HashGrid]:
        a = (self.hash_levels, self.hash_features, self.hash_log2_size, self.hash_base_res, self.hash_scale)
        return [HashGrid(3, *a), HashGrid(2, *a)]

    @property
    def n_in(self) -> int:
        if self.encoding == ENC_HASHGRID:
            return 2 * self.hash_levels * self.hash_features + 1
        return 12 * self.in_freqs

    def shapes(self) -> List[Tuple[int, int]]:
        s = [(self.hidden, self.n_in)]
        s += [(self.hidden, self.hidden)] * (self.n_hidden - 1)
        s += [(3, self.hidden)]
        return s

    def n_mlp(self) -> int:
        return sum(o * i for o, i in self.shapes())

    def n_params(self) -> int:
        n = self.n_mlp()
        if self.encoding == ENC_HASHGRID:
            n = (n + 7) // 8 * 8 + sum(g.n_params() for g in self.grids())
        return n

    def table_offsets(self) -> List[List[int]]:
        """Float offset of every level's table in the flat parameter vector:
        after the MLP layers (rounded up to 8 floats), position grid levels,
        then direction grid levels."""
        o = (self.n_mlp() + 7) // 8 * 8
        out = []
        for g in self.grids():
            offs = []
            for l in range(g.levels):
                offs.append(o)
                o += g.level_floats(l)
            out.append(offs)
        return out


def unflatten(flat: np.ndarray, desc: FieldDesc) -> List[np.ndarray]:
    """The MLP layers' weight matrices (hash tables, if any, are not part of it)."""
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
    w = (2u - 1) sqrt(6/fan_in) evaluated in FP64, then rounded once.  Hash
    tables: element e of level l of grid j (0 position, 1 direction) draws u
    from item 64 + 16 j + l: w = (2u - 1) 1e-4; padding floats are 0."""
    from . import philox_item, philox_stream, uniform, TAG_INIT
    flat = []
    for l, (o, i) in enumerate(desc.shapes()):
        n = o * i
        nb = (n + 3) // 4
        words = philox_stream(desc.seed, TAG_INIT, 0, l + 1, nb)[l]
        u = uniform(words.reshape(-1)[:n])
        bound = math.sqrt(6.0 / i)
        flat.append(((2.0 * u - 1.0) * bound).astype(np.float32))
    w = np.concatenate(flat)
    if desc.encoding != ENC_HASHGRID:
        return w
    out = np.zeros(desc.n_params(), np.float32)
    out[:w.size] = w
    for j, (g, offs) in enumerate(zip(desc.grids(), desc.table_offsets())):
        for l in range(g.levels):
            n = g.entries(l) * g.features
            nb = (n + 3) // 4
            words = philox_item(desc.seed, TAG_INIT, 0, 64 + 16 * j + l, nb)
            u = uniform(words.reshape(-1)[:n])
            out[offs[l]:offs[l] + n] = ((2.0 * u - 1.0) * HASH_INIT).astype(np.float32)
    return out


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
    return f.reshape(q.shape[0], q.shape[1] * n_freq * 2)      # also for an empty batch


def hash_corners(grid: HashGrid, l: int, x: np.ndarray):
    """Table indices (B, 2^dim) and interpolation weights (B, 2^dim) of level
    l at points x (B, dim).  The cell is decided in float32, as the kernel
    does: p = float32(clamp(x, 0, 1)) * N_l, i = min(floor(p), N_l - 1),
    fraction p - i (exact in float32); corner c takes vertex i + c with weight
    prod_k (c_k ? f_k : 1 - f_k) (multilinear interpolation)."""
    N = grid.res(l)
    xc = np.clip(np.asarray(x, np.float32), np.float32(0), np.float32(1))
    p = xc * np.float32(N)
    i = np.minimum(np.floor(p), np.float32(N - 1)).astype(np.int64)
    f = (p - i.astype(np.float32)).astype(np.float64)
    B, d = xc.shape
    idx = np.zeros((B, 2 ** d), np.int64)
    wgt = np.ones((B, 2 ** d))
    for c in range(2 ** d):
        v = [i[:, k] + ((c >> k) & 1) for k in range(d)]
        for k in range(d):
            wgt[:, c] *= np.where((c >> k) & 1, f[:, k], 1.0 - f[:, k])
        if grid.dense(l):
            lin = np.zeros(B, np.int64)
            for k in range(d - 1, -1, -1):
                lin = lin * (N + 1) + v[k]
            idx[:, c] = lin
        else:
            h = np.zeros(B, np.uint64)
            for k in range(d):
                h ^= (v[k].astype(np.uint64) * np.uint64(HASH_PRIMES[k])) & np.uint64(0xFFFFFFFF)
            idx[:, c] = (h & np.uint64(2 ** grid.log2_size - 1)).astype(np.int64)
    return idx, wgt


def hash_encode(weights: np.ndarray, q: np.ndarray, desc: FieldDesc):
    """Hash-grid input of the MLP: [position levels' features, direction
    levels' features, g], level-major, F features per level.  Returns the
    (B, n_in) inputs and the corner lists for the backward pass."""
    q = np.asarray(q, np.float64)
    w = np.asarray(weights, np.float64)
    B = q.shape[0]
    cols, corners = [], []
    for j, (g, offs) in enumerate(zip(desc.grids(), desc.table_offsets())):
        x = q[:, 0:3] if j == 0 else q[:, 3:5]
        for l in range(g.levels):
            idx, wgt = hash_corners(g, l, x)
            F = g.features
            tab = w[offs[l]:offs[l] + g.entries(l) * F].reshape(-1, F)
            cols.append(np.einsum("bc,bcf->bf", wgt, tab[idx]))
            corners.append((offs[l], F, idx, wgt))
    cols.append(q[:, 5:6])
    return np.concatenate(cols, 1).reshape(B, -1), corners


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
    corners = None
    if desc.encoding == ENC_HASHGRID:
        h, corners = hash_encode(weights, q, desc)
    elif desc.prec == PREC_F32:
        h = encode(q, desc.in_freqs)
    else:
        # the tensor-core fields compute the features in float32 before
        # rounding them to the operand type: the rounding is taken on the
        # same float32 values (within a few 1e-6 of sin / cos, see encode_f32)
        from . import encode_f32
        h = encode_f32(q, desc.in_freqs)
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
    return h, (ins, zs, corners)


def backward(weights: np.ndarray, cache, dy: np.ndarray, desc: FieldDesc) -> np.ndarray:
    """dW = sum_b (d yhat_b / dW)^T dy_b for every layer, flattened; for a
    hash-grid field also the tables' gradient: the MLP input's gradient
    d_in = d_0 W_0 (W_0 as the forward used it, the input's rounding taken as
    the identity) spread over each level's corners with their interpolation
    weights."""
    ws = unflatten(weights, desc)
    ins, zs, corners = cache
    L = len(ws)
    grads = [None] * L
    d = np.asarray(dy, np.float64)
    for l in range(L - 1, -1, -1):
        grads[l] = d.T @ ins[l]
        if l == 0:
            if corners is not None:
                W0 = ws[0] if L == 1 else rnd(ws[0], desc.prec)
                d_in = d @ W0
                out = np.zeros(desc.n_params())
                mlp = flatten(grads)
                out[:mlp.size] = mlp
                col = 0
                for off, F, idx, wgt in corners:
                    contrib = wgt[:, :, None] * d_in[:, None, col:col + F]
                    tgt = off + idx[:, :, None] * F + np.arange(F)[None, None, :]
                    np.add.at(out, tgt.reshape(-1), contrib.reshape(-1))
                    col += F
                return out
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


def train_gradient(weights: np.ndarray, q: np.ndarray, y: np.ndarray, desc: FieldDesc, scales=None):
    """The training step's loss and gradient (Sec. 3.5.1): the mean relative
    MSE of the forward pass against targets y, and its gradient with loss
    scaling -- the backward pass runs on n times the gradient of the mean
    (n = the number of outputs), 2 (yhat - y) / (y^2 + eps) per output, so
    that its gradients rounded to a 16-bit field precision keep their
    significant bits, and the result is divided by n.  In FP64 without
    rounding (PREC_F32) the scaling is exact: the result is the plain
    gradient of the mean."""
    yh, cache = forward(weights, q, desc, scales)
    loss, dy = rel_mse(yh, y)
    n = yh.size
    return loss, backward(weights, cache, dy * n, desc) / n


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
