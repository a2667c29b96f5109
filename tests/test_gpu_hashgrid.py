"""GPU parity of the hash-grid photon field (Sec. 3.4) against the oracle.

  * seeded initialisation of the MLP and the level tables: bit-identical;
  * forward L' at oracle-generated queries (tables set to oracle-drawn values
    large enough for the encoding to matter): float32 within 1e-5, bf16 /
    fp16 within 2e-2 of the precision-emulated oracle;
  * backward: every MLP layer's and every level table's gradient within
    1e-5 (f32) / 1e-3 (bf16, f16) norm-wise; the oracle's gradient is pinned
    by central differences (tests/test_oracle_hashgrid.py);
  * training on photon-cache targets lowers the loss;
  * a hash-grid field renders (march mode) within the float32-field bars;
  * invalid descriptions are refused.
Levels are dense and hashed in every configuration; the cell of each level
is decided in float32 on both sides.
"""
import math

import numpy as np
import pytest
import torch

from oracle import field as F
from paper_2304_07338_b300 import api, inputs as I

pytestmark = pytest.mark.gpu

PRECS = {"f32": F.PREC_F32, "bf16": F.PREC_BF16, "f16": F.PREC_F16}
# hidden, n_hidden, levels, features, log2 table size, base resolution, scale
CONFIGS = {
    "small": (32, 2, 4, 2, 10, 4, 2.0),
    "odd_scale": (64, 3, 6, 8, 12, 3, 1.5),
    "paper_levels": (64, 4, 16, 8, 14, 16, 2.0),
}


def _pair(ctx, cfg, prec="f32", seed=11):
    h, nh, L, Fe, T, b, s = CONFIGS[cfg]
    fld = api.Field(ctx, 12, h, nh, prec, 5.0, seed=seed, encoding="hashgrid", hash_levels=L, hash_features=Fe,
                    hash_log2_size=T, hash_base_res=b, hash_scale=s)
    desc = F.FieldDesc(12, h, nh, PRECS[prec], 5.0, seed, F.ENC_HASHGRID, L, Fe, T, b, s)
    return fld, desc


def _queries(n, seed=0):
    rng = np.random.default_rng(seed)
    q = rng.uniform(0, 1, (n, 6))
    q[:5, :3] = [[0, 0, 0], [1, 1, 1], [0.5, 0.25, 1.0], [1e-7, 0.999999, 0.5], [0.75, 0.75, 0.75]]
    q[:, 5] = rng.choice([-0.5, 0.0, 0.5], n)
    return q.astype(np.float32)


def _loud_tables(w, desc, seed=1):
    # oracle-drawn table values of order 0.3, so that the encoding moves L'
    w = w.astype(np.float64).copy()
    rng = np.random.default_rng(seed)
    n0 = (desc.n_mlp() + 7) // 8 * 8
    w[n0:] = rng.normal(size=w.size - n0) * 0.3
    return w.astype(np.float32)


@pytest.mark.parametrize("cfg", sorted(CONFIGS))
def test_init_bit_identical(pf_ctx, cfg):
    fld, desc = _pair(pf_ctx, cfg)
    w = F.init_weights(desc)
    assert fld.n_params == desc.n_params() == w.size
    assert np.array_equal(fld.get_weights().cpu().numpy(), w)
    g = desc.grids()
    assert any(g[0].dense(l) for l in range(g[0].levels)) and any(not g[0].dense(l) for l in range(g[0].levels))


@pytest.mark.parametrize("cfg,prec,tol", [("small", "f32", 1e-5), ("odd_scale", "f32", 1e-5),
                                          ("paper_levels", "f32", 1e-5), ("odd_scale", "bf16", 2e-2),
                                          ("paper_levels", "f16", 2e-2)])
def test_forward_matches_oracle(pf_ctx, cfg, prec, tol):
    fld, desc = _pair(pf_ctx, cfg, prec)
    w = _loud_tables(F.init_weights(desc), desc)
    fld.set_weights(torch.from_numpy(w).cuda())
    q = _queries(1000 + 37)
    y = fld.forward(torch.from_numpy(q).cuda()).cpu().numpy()
    ref, _ = F.forward(w.astype(np.float64), q.astype(np.float64), desc)
    assert np.abs(y - ref).max() <= tol, np.abs(y - ref).max()
    # the tables matter: zeroing them moves the output by far more than the bar
    w0 = w.copy()
    w0[(desc.n_mlp() + 7) // 8 * 8:] = 0
    ref0, _ = F.forward(w0.astype(np.float64), q.astype(np.float64), desc)
    assert np.abs(ref0 - ref).max() > 20 * tol


@pytest.mark.parametrize("cfg,prec", [("small", "f32"), ("odd_scale", "f32"), ("paper_levels", "f32"),
                                      ("odd_scale", "bf16"), ("small", "f16"), ("paper_levels", "bf16"),
                                      ("paper_levels", "f16")])
def test_backward_matches_oracle(pf_ctx, cfg, prec):
    fld, desc = _pair(pf_ctx, cfg, prec, seed=4)
    w = _loud_tables(F.init_weights(desc), desc, seed=2)
    fld.set_weights(torch.from_numpy(w).cuda())
    q = _queries(512, seed=3)
    dy = np.random.default_rng(5).normal(size=(512, 3)).astype(np.float32)
    dw = fld.backward(torch.from_numpy(q).cuda(), torch.from_numpy(dy).cuda()).cpu().numpy().astype(np.float64)
    _, cache = F.forward(w.astype(np.float64), q.astype(np.float64), desc)
    ref = F.backward(w.astype(np.float64), cache, dy.astype(np.float64), desc)
    bar = 1e-5 if prec == "f32" else 1e-3
    for a, b in zip(F.unflatten(dw, desc), F.unflatten(ref, desc)):
        assert np.linalg.norm(a - b) <= bar * np.linalg.norm(b)
    for j, (g, offs) in enumerate(zip(desc.grids(), desc.table_offsets())):
        for l in range(g.levels):
            sl = slice(offs[l], offs[l] + g.level_floats(l))
            nb = np.linalg.norm(ref[sl])
            assert nb > 0
            assert np.linalg.norm(dw[sl] - ref[sl]) <= bar * nb, (j, l)


def test_training_reduces_loss(pf_ctx, orc):
    sc = I.scene_judge(32)
    vol = api.Volume.from_inputs(sc.volume)
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, sc.g_set, 20000, 16, 16, seed=3)
    fld = api.Field(pf_ctx, 12, 64, 3, "bf16", 5.0, seed=8, encoding="hashgrid", hash_levels=8, hash_features=4,
                    hash_log2_size=14, hash_base_res=4, hash_scale=1.5)
    loss = fld.train(cache, steps=60, batch=4096, lr=1e-2, seed=3)
    assert np.all(np.isfinite(loss))
    assert loss[-10:].mean() < 0.5 * loss[:5].mean(), (loss[:5], loss[-10:])


def test_march_render_with_hashgrid_field(pf_ctx, orc):
    sc = I.scene_small(64, 64, 64, 4)
    vol = api.Volume.from_inputs(sc.volume)
    fld, desc = _pair(pf_ctx, "odd_scale", "f32", seed=3)
    w = _loud_tables(F.init_weights(desc), desc, seed=7)
    fld.set_weights(torch.from_numpy(w).cuda())
    img = api.render_neural(pf_ctx, vol, sc.lights, sc.g, sc.camera, sc.spp, 0.5, seed=5, field=fld)
    pf_ctx.sync()
    # the oracle's float32 instantiation: the same interaction points and
    # float32 field queries, so every level's cell is the same on both sides;
    # the field in FP64.  Each pixel within what the float32 field's L'
    # tolerance (1e-5) allows, plus float rounding of the direct part.
    ref, cs, Li = orc.render_neural(sc.volume, sc.lights, sc.g, sc.camera, sc.spp, 0.5, 5,
                                    weights=w.astype(np.float64), desc=desc, fp32=True, return_parts=True)
    assert Li.max() > 0
    ali = (cs["albedo"] * Li).sum(axis=2) / sc.spp
    direct = (cs["albedo"] * cs["Ld"]).sum(axis=2) / sc.spp
    d = np.abs(img.cpu().numpy().astype(np.float64) - ref)
    bound = math.expm1(5.0 * math.log(10.0) * 1e-5) * ali + 2e-6 * np.maximum(np.abs(ref), 1e-3 * direct.max())
    assert np.all(d <= bound + 1e-30), (d / (bound + 1e-30)).max()


def test_invalid_descriptions(pf_ctx):
    bad = [dict(prec="fp8"), dict(hash_levels=0), dict(hash_levels=17), dict(hash_features=3),
           dict(hash_log2_size=25), dict(hash_scale=5.0), dict(hash_base_res=0),
           dict(hash_base_res=65536, hash_levels=16)]
    for kw in bad:
        args = dict(prec="f32", encoding="hashgrid", hash_levels=4, hash_features=2, hash_log2_size=10,
                    hash_base_res=4, hash_scale=2.0)
        args.update(kw)
        with pytest.raises(api.PfError):
            api.Field(pf_ctx, 12, 32, 2, args.pop("prec"), 5.0, seed=1, **args)
