"""GPU parity of the field network, its training samples and training
(Sec. 3.3-3.5) against the oracle, through the C ABI.

  * seeded Kaiming-uniform initialisation: bit-identical weights;
  * forward L' at oracle-generated queries: float32 field within 1e-5;
    bf16 / fp16 / fp8 fields within 2e-2 of the precision-emulated oracle;
  * backward: per-layer gradient error <= 1e-3 (relative, norm-wise) against
    the precision-emulated oracle on a 512-query batch, and the oracle's own
    gradient is pinned by finite differences (tests/test_oracle_field.py);
    the training loss and its loss-scaled gradient likewise on 4133 queries;
  * Adam step against the closed form;
  * training queries: identical cells and g, positions and angles within
    float32 rounding; radiance estimates within 1e-5 (float32 sums of the
    same records);
  * training lowers the loss.
"""
import numpy as np
import pytest
import torch

from oracle import field as F
from paper_2304_07338_b300 import api, inputs as I

pytestmark = pytest.mark.gpu

PRECS = {"f32": F.PREC_F32, "bf16": F.PREC_BF16, "f16": F.PREC_F16, "fp8": F.PREC_FP8}


def _queries(n, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0, 1, (n, 6))
    q[:, 5] = rng.choice([-0.5, 0.0, 0.5], n)
    return q.astype(np.float32)


@pytest.mark.parametrize("prec,hidden,n_hidden,tol", [("f32", 64, 3, 1e-5), ("bf16", 64, 4, 2e-2),
                                                     ("f16", 64, 4, 2e-2), ("f16", 128, 4, 2e-2),
                                                     ("fp8", 128, 4, 2e-2)])
def test_forward_matches_emulated_oracle(pf_ctx, prec, hidden, n_hidden, tol):
    fld = api.Field(pf_ctx, 12, hidden, n_hidden, prec, 5.0, seed=21)
    desc = F.FieldDesc(12, hidden, n_hidden, PRECS[prec], 5.0, 21)
    w = F.init_weights(desc)
    assert np.array_equal(fld.get_weights().cpu().numpy(), w)
    q = _queries(1000 + 37)                  # several 128-row tiles and a ragged tail
    qt = torch.from_numpy(q).cuda()
    scales = None
    if prec == "fp8":
        cal = _queries(4096, seed=9)
        fld.calibrate_fp8(torch.from_numpy(cal).cuda())
        scales = F.fp8_calibrate(w.astype(np.float64), cal.astype(np.float64), desc)
    y = fld.forward(qt).cpu().numpy()
    ref, _ = F.forward(w.astype(np.float64), q.astype(np.float64), desc, scales)
    err = np.abs(y - ref)
    assert err.max() <= tol, err.max()
    if prec != "f32":
        # the unquantised network differs by more than the emulation tolerance
        ref32, _ = F.forward(w.astype(np.float64), q.astype(np.float64), F.FieldDesc(12, hidden, n_hidden, 0, 5.0, 21))
        assert np.abs(ref32 - ref).max() > 0


def test_forward_empty_and_single(pf_ctx):
    fld = api.Field(pf_ctx, 12, 64, 3, "f32", 5.0, seed=1)
    y = fld.forward(torch.zeros(0, 6, device="cuda"))
    assert y.shape == (0, 3)
    q = _queries(1)
    y1 = fld.forward(torch.from_numpy(q).cuda()).cpu().numpy()
    desc = F.FieldDesc(12, 64, 3, 0, 5.0, 1)
    ref, _ = F.forward(F.init_weights(desc).astype(np.float64), q.astype(np.float64), desc)
    assert np.abs(y1 - ref).max() < 1e-5


@pytest.mark.parametrize("prec,hidden", [("f32", 64), ("bf16", 64), ("f16", 64), ("f16", 128), ("bf16", 128)])
def test_backward_matches_oracle(pf_ctx, prec, hidden):
    n_hidden = 4
    fld = api.Field(pf_ctx, 12, hidden, n_hidden, prec, 5.0, seed=4)
    desc = F.FieldDesc(12, hidden, n_hidden, PRECS[prec], 5.0, 4)
    w = F.init_weights(desc).astype(np.float64)
    q = _queries(512, seed=3)
    dy = np.random.default_rng(5).normal(size=(512, 3)).astype(np.float32)
    dw = fld.backward(torch.from_numpy(q).cuda(), torch.from_numpy(dy).cuda()).cpu().numpy()
    _, cache = F.forward(w, q.astype(np.float64), desc)
    ref = F.backward(w, cache, dy.astype(np.float64), desc)
    for (a, b) in zip(F.unflatten(dw, desc), F.unflatten(ref, desc)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= (1e-5 if prec == "f32" else 1e-3), rel


@pytest.mark.parametrize("prec,hidden", [("f32", 64), ("bf16", 64), ("f16", 128), ("bf16", 128)])
def test_loss_gradient_matches_oracle(pf_ctx, prec, hidden):
    """The training step's loss and gradient (Sec. 3.5.1; the backward pass
    loss-scaled as in training) against the precision-emulated oracle on
    4133 queries (several tiles of either tensor-core trainer and a ragged
    tail) with targets near the prediction: loss within 1e-5 (f32) / 1e-3
    (16-bit) relative, gradient within 1e-5 / 1e-3 norm-wise per layer."""
    fld = api.Field(pf_ctx, 12, hidden, 4, prec, 5.0, seed=6)
    desc = F.FieldDesc(12, hidden, 4, PRECS[prec], 5.0, 6)
    w = F.init_weights(desc).astype(np.float64)
    q = _queries(4133, seed=12)
    y0, _ = F.forward(w, q.astype(np.float64), F.FieldDesc(12, hidden, 4, F.PREC_F32, 5.0, 6))
    t = (y0 + np.random.default_rng(13).normal(size=y0.shape) * 0.3).astype(np.float32)
    loss, dw = fld.loss_gradient(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda())
    lref, gref = F.train_gradient(w, q.astype(np.float64), t.astype(np.float64), desc)
    tol = 1e-5 if prec == "f32" else 1e-3
    assert abs(loss - lref) <= tol * lref, (loss, lref)
    for a, b in zip(F.unflatten(dw.cpu().numpy(), desc), F.unflatten(gref, desc)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= tol, rel


@pytest.mark.parametrize("prec,hidden,n", [("bf16", 64, 77), ("bf16", 64, 257), ("f16", 128, 33), ("f16", 128, 65)])
def test_loss_gradient_partial_tiles(pf_ctx, prec, hidden, n):
    """The tensor-core trainers on batches that end inside a tile (one
    partial tile only, or one row past whole tiles): rows past the batch must
    add nothing to the loss or any weight gradient (including the output
    layer's, summed from registers), and the next tile's inputs are loaded
    ahead past the end.  Same bars as the full test."""
    fld = api.Field(pf_ctx, 12, hidden, 4, prec, 5.0, seed=9)
    desc = F.FieldDesc(12, hidden, 4, PRECS[prec], 5.0, 9)
    w = F.init_weights(desc).astype(np.float64)
    q = _queries(n, seed=21)
    y0, _ = F.forward(w, q.astype(np.float64), F.FieldDesc(12, hidden, 4, F.PREC_F32, 5.0, 9))
    t = (y0 + np.random.default_rng(22).normal(size=y0.shape) * 0.3).astype(np.float32)
    loss, dw = fld.loss_gradient(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda())
    lref, gref = F.train_gradient(w, q.astype(np.float64), t.astype(np.float64), desc)
    assert abs(loss - lref) <= 1e-3 * lref, (loss, lref)
    for a, b in zip(F.unflatten(dw.cpu().numpy(), desc), F.unflatten(gref, desc)):
        rel = np.linalg.norm(a - b) / np.linalg.norm(b)
        assert rel <= 1e-3, rel


def test_autograd_function(pf_ctx):
    fld = api.Field(pf_ctx, 12, 64, 3, "f32", 5.0, seed=2)
    w = fld.get_weights().clone().requires_grad_(True)
    q = torch.from_numpy(_queries(300)).cuda()
    y = api.FieldFunction.apply(fld, q, w)
    (y * y).sum().backward()
    dw = fld.backward(q, (2 * y).detach())
    # float32 atomics make the block-sum order vary between calls
    assert torch.allclose(w.grad, dw, rtol=1e-4, atol=1e-6)


def test_adam_step(pf_ctx):
    fld = api.Field(pf_ctx, 12, 64, 3, "f32", 5.0, seed=2)
    w0 = F.init_weights(F.FieldDesc(12, 64, 3, F.PREC_F32, 5.0, 2)).astype(np.float64)   # the field's seeded init
    g = np.random.default_rng(1).normal(size=w0.size).astype(np.float32)
    fld.adam(torch.from_numpy(g).cuda(), 1e-2, 0.9, 0.99, 1e-8)
    w1 = fld.get_weights().cpu().numpy()
    want, _, _ = F.adam_step(w0, 0 * w0, 0 * w0, g.astype(np.float64), 1, 1e-2, 0.9, 0.99, 1e-8)
    assert np.abs(w1 - want).max() < 1e-6


@pytest.fixture(scope="module")
def small_cache(pf_ctx, orc):
    sc = I.scene_judge(32)
    vol = api.Volume.from_inputs(sc.volume)
    res = 16
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, sc.g_set, 20000, 16, res, seed=3)
    tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, 20000, 16, res, seed=3, fp32=True)
    oc = orc.build_cache(tr)
    csig = orc.cell_sigma(sc.volume, res)
    return sc, cache, oc, csig


def test_query_sampler_matches_oracle(pf_ctx, orc, small_cache):
    sc, cache, oc, csig = small_cache
    occ = orc.occupied_cells(oc, csig)
    B = 4099
    qg = cache.sample_queries(B, step=7, seed=99).cpu().numpy()
    qo, gi = orc.sample_queries(occ, 16, sc.g_set, B, 7, 99)
    np.testing.assert_allclose(qg[:, :3], qo[:, :3], rtol=0, atol=2e-7)
    np.testing.assert_allclose(qg[:, 3:5], qo[:, 3:5], rtol=0, atol=2e-6)
    assert np.array_equal(qg[:, 5], qo[:, 5].astype(np.float32))


def test_targets_match_oracle(pf_ctx, orc, small_cache):
    sc, cache, oc, csig = small_cache
    occ = orc.occupied_cells(oc, csig)
    q, _ = orc.sample_queries(occ, 16, sc.g_set, 3000, 0, 5)
    q32 = q.astype(np.float32)
    ls, lp = cache.estimate_targets(torch.from_numpy(q32).cuda(), 5.0)
    ref = orc.estimate_targets(q32.astype(np.float64), sc.g_set, oc, csig)
    np.testing.assert_allclose(ls.cpu().numpy(), ref, rtol=2e-5, atol=1e-30)
    np.testing.assert_allclose(lp.cpu().numpy(), F.log_encode(ref, 5.0), rtol=0, atol=2e-6)


@pytest.mark.parametrize("prec,hidden", [("f32", 64), ("bf16", 64), ("f16", 128)])
def test_training_reduces_loss(pf_ctx, small_cache, prec, hidden):
    sc, cache, oc, csig = small_cache
    fld = api.Field(pf_ctx, 12, hidden, 4, prec, 5.0, seed=8)
    loss = fld.train(cache, steps=60, batch=4096, lr=1e-2, seed=3)
    assert np.all(np.isfinite(loss))
    assert loss[-10:].mean() < 0.5 * loss[:5].mean(), (loss[:5], loss[-10:])


@pytest.mark.parametrize("freqs", [12, 7, 16, 1])
def test_encoding_matches_float32_oracle(pf_ctx, freqs):
    """pf_field_encode (Sec. 3.4's gamma in the tensor-core fields' float32
    steps) is bit-identical to the oracle's float32 encoding, on several
    launch blocks with a ragged tail and on edge inputs (0, 1, 1/2, values
    just below 1, negative g, a denormal)."""
    import oracle
    q = _queries(3 * 256 + 41, seed=5)
    edge = np.array([[0.0, 1.0, 0.5, 0.25, np.nextafter(np.float32(1), np.float32(0)), -0.75],
                     [1e-40, 0.999, 0.125, 0.75, 0.3333333, 0.9],
                     [0.5, 0.0, 1.0, 0.0625, 0.1, -0.9]], np.float32)
    q = np.concatenate([q, edge]).astype(np.float32)
    got = api.field_encode(pf_ctx, torch.from_numpy(q).cuda(), freqs).cpu().numpy()
    ref = oracle.encode_f32(q, freqs)
    assert got.shape == (q.shape[0], 12 * freqs)
    assert np.array_equal(got.astype(np.float64), ref)
    # and within the pinned accuracy of the exact features
    k = np.arange(freqs)
    a = np.pi * (2.0 ** k)[None, None, :] * q.astype(np.float64)[:, :, None]
    exact = np.stack([np.sin(a), np.cos(a)], axis=3).reshape(q.shape[0], 12 * freqs)
    assert np.abs(got - exact).max() < 6e-6


def test_encoding_refuses_bad_arguments(pf_ctx):
    q = torch.zeros(6, dtype=torch.float32, device="cuda")
    out = torch.zeros(12, dtype=torch.float32, device="cuda")
    lib = pf_ctx.lib
    assert lib.pf_field_encode(pf_ctx.h, q.data_ptr(), 1, 0, out.data_ptr()) == 1
    assert lib.pf_field_encode(pf_ctx.h, q.data_ptr(), 1, 17, out.data_ptr()) == 1
    assert lib.pf_field_encode(pf_ctx.h, q.data_ptr(), -1, 1, out.data_ptr()) == 1
    assert lib.pf_field_encode(pf_ctx.h, None, 1, 1, out.data_ptr()) == 1
    assert lib.pf_field_encode(pf_ctx.h, q.data_ptr(), 0, 1, None) == 0     # empty batch: no-op
    assert api.field_encode(pf_ctx, torch.zeros((0, 6), dtype=torch.float32, device="cuda")).shape == (0, 144)
