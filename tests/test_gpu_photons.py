"""GPU parity of photon tracing (Algorithm 1) and the photon caches.

The tracer's float32 arithmetic follows the same IEEE operations as the
oracle's float32 instantiation, so every record -- its cache bin, its photon
id and interaction index, its direction and its power -- is bit-identical,
and so are the per-key counts.  Per-key power sums are FP64 sums in an order
the GPU does not fix; they agree with the oracle's to one float32 ulp.
At the full data-source size (2^20 photons per light per g) the oracle traces
sampled photon-id ranges and the GPU records of those photons must match.
"""
import numpy as np
import pytest
import torch

from paper_2304_07338_b300 import api, inputs as I

pytestmark = pytest.mark.gpu


def _gpu_records(cache):
    ex = cache.export()
    rid = ex["id"].cpu().numpy().view(np.uint32).astype(np.int64)
    order = np.argsort(rid, kind="stable")
    return dict(id=rid[order], key=ex["key"].cpu().numpy().view(np.uint32)[order],
                dir=ex["dir"].cpu().numpy()[order], phi=ex["phi"].cpu().numpy()[order],
                counts=ex["counts"].cpu().numpy().view(np.uint32), flux=ex["flux"].cpu().numpy(),
                occupied=ex["occupied"].cpu().numpy().view(np.uint32), cell_sigma=ex["cell_sigma"].cpu().numpy())


def _oracle_records(tr):
    S = tr["keys"].shape[1]
    mask = np.arange(S)[None, :] < tr["nrec"][:, None]
    pid = np.broadcast_to((np.arange(tr["keys"].shape[0]) + tr["p_begin"])[:, None], mask.shape)
    slot = np.broadcast_to(np.arange(S)[None, :], mask.shape)
    rid = (pid[mask].astype(np.int64) << 4) | slot[mask]
    return dict(id=rid, key=tr["keys"][mask], dir=tr["dirs"][mask], phi=tr["phis"][mask])


@pytest.mark.parametrize("use_rr", [True, False])
def test_records_bit_exact(pf_ctx, orc, use_rr):
    sc = I.scene_judge(32)
    vol = api.Volume.from_inputs(sc.volume)
    N, res = 5000, 16
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, sc.g_set, N, 16, res, seed=77, use_rr=use_rr)
    g = _gpu_records(cache)
    tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, N, 16, res, seed=77, use_rr=use_rr, fp32=True)
    o = _oracle_records(tr)
    assert g["id"].size == o["id"].size == cache.n_records
    assert np.array_equal(g["id"], o["id"])
    assert np.array_equal(g["key"], o["key"])
    assert np.array_equal(g["dir"].view(np.uint32), o["dir"].view(np.uint32))
    assert np.array_equal(g["phi"].view(np.uint32), o["phi"].view(np.uint32))
    oc = orc.build_cache(tr)
    assert np.array_equal(g["counts"].astype(np.int64), oc["counts"])
    np.testing.assert_allclose(g["flux"], oc["cache"], rtol=2 ** -23, atol=0)
    assert np.allclose(cache.tally(), tr["tally"], rtol=1e-12, atol=0)
    csig = orc.cell_sigma(sc.volume, res)
    np.testing.assert_allclose(g["cell_sigma"], csig, rtol=1e-5, atol=1e-6)
    assert np.array_equal(g["occupied"].astype(np.int64), orc.occupied_cells(oc, csig))


def test_directional_light_and_small_bounce_cap(pf_ctx, orc):
    sc = I.scene_small(32)
    vol = api.Volume.from_inputs(sc.volume)
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, (-0.75, 0.75), 3000, 3, 8, seed=5)
    g = _gpu_records(cache)
    tr = orc.trace_photons(sc.volume, sc.lights, (-0.75, 0.75), 3000, 3, 8, seed=5, fp32=True)
    o = _oracle_records(tr)
    assert np.array_equal(g["id"], o["id"]) and np.array_equal(g["key"], o["key"])
    assert np.array_equal(g["phi"].view(np.uint32), o["phi"].view(np.uint32))
    assert np.all((g["id"] & 15) < 2)          # at most interactions 2 and 3


def test_full_size_sampled_photons(pf_ctx, orc):
    """Data-source workload (128^3 fBm, 2 point lights, G = {-0.5, 0, 0.5},
    2^20 photons per light per g, 64^3 caches): GPU records of sampled photon
    id ranges equal the oracle's, computed photon by photon."""
    sc = I.scene_judge()
    vol = api.Volume.from_inputs(sc.volume)
    N = 1 << 20
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, sc.g_set, N, 16, 64, seed=20230415)
    assert cache.info.n_photons == 6 * N
    g = _gpu_records(cache)
    assert g["counts"].sum() == cache.n_records
    P = 6 * N
    for p0 in (0, N + 12345, 3 * N - 4000, P - 4000):
        tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, N, 16, 64, seed=20230415, fp32=True,
                               p_begin=p0, p_end=p0 + 4000)
        o = _oracle_records(tr)
        lo, hi = np.searchsorted(g["id"], [p0 << 4, (p0 + 4000) << 4])
        assert np.array_equal(g["id"][lo:hi], o["id"])
        assert np.array_equal(g["key"][lo:hi], o["key"])
        assert np.array_equal(g["phi"][lo:hi].view(np.uint32), o["phi"].view(np.uint32))
    t = cache.tally()
    assert np.allclose(t[0], t[1:].sum(0), rtol=1e-9)


def test_brick_majorants_match_oracle(pf_ctx, orc):
    for n, tf, dt, B in ((32, I.tf_white_alpha_ramp(), np.float32, 8), (40, I.tf_piecewise_rgba(64), np.float16, 8),
                         (27, I.tf_piecewise_rgba(256), np.uint8, 8), (40, I.tf_piecewise_rgba(64), np.float32, 16),
                         (37, I.tf_white_alpha_ramp(), np.uint8, 4), (70, I.tf_piecewise_rgba(64), np.float16, 32),
                         (150, I.tf_white_alpha_ramp(), np.uint8, 64)):
        data = I.fbm_volume(n, seed=n)
        if dt == np.uint8:
            data = np.round(data * 255).astype(np.uint8)
        else:
            data = data.astype(dt)
        v = I.Volume(data, 17.0, 0.9, tf, brick=B)
        g = api.Volume.from_inputs(v).brick_majorants(pf_ctx).cpu().numpy()
        want = orc.brick_majorants(v, fp32=True).astype(np.float32)
        assert g.shape == want.shape and np.array_equal(g.view(np.uint32), want.view(np.uint32))


def test_invalid_arguments(pf_ctx):
    sc = I.scene_small(8)
    vol = api.Volume.from_inputs(sc.volume)
    with pytest.raises(api.PfError):
        api.build_photon_cache(pf_ctx, vol, sc.lights, (0.0,), 100, 16, 48)      # res not a power of two
    with pytest.raises(api.PfError):
        api.build_photon_cache(pf_ctx, vol, sc.lights, (1.0,), 100, 16, 8)       # |g| >= 1
    with pytest.raises(api.PfError):
        api.build_photon_cache(pf_ctx, vol, sc.lights, (0.0,), 0, 16, 8)         # no photons
