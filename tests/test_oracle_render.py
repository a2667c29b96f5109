"""Pins of the oracle's renderers (Algorithm 2 and the path-tracing baseline).

Closed form: a homogeneous box lit by a directional light along the view axis
and seen by a near-orthographic camera from the light's side.  Single
scattering gives the pixel value A p_g(-1) E (1 - exp(-2 sigma)) / 2; the
ray-marched renderer, the delta/ratio-tracking renderer and the path tracer
limited to one bounce must all converge to it.  Per sample, the marched
renderer's free flight inverts exp(-sigma t) exactly and its shadow rays obey
Beer-Lambert exactly.  The one-bounce path tracer and the field-less neural
renderer in tracking mode are the same estimator on the same random numbers.
Multi-bounce: the neural renderer fed with the photon-map estimate of the
indirect in-scattered radiance (photons traced by Algorithm 1) matches the
full path tracer up to the grid estimator's bias.
"""
import math

import numpy as np
import pytest

from paper_2304_07338_b300 import inputs as I


SIGMA, ALB, G = 1.5, 0.8, 0.5


def _setup(W=2, H=2):
    vol = I.Volume(np.ones((8, 8, 8), np.float32), SIGMA, ALB, I.tf_constant(1.0))
    light = I.Light(I.DIRECTIONAL, (0.0, 0.0, 1.0), (1.0, 1.0, 1.0))
    cam = I.Camera((0.5, 0.5, 100.0), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.01, W, H)
    return vol, [light], cam


def _closed_form():
    p = (1 - G * G) / (1 + G) ** 3 / (4 * math.pi)      # p_g(mu = -1)
    return ALB * p * (1 - math.exp(-2 * SIGMA)) / 2


def _mean_se(x):
    x = np.asarray(x).reshape(-1)
    return x.mean(), x.std(ddof=1) / math.sqrt(x.size)


@pytest.mark.parametrize("fp32", [False, True])
def test_march_free_flight_and_beer_lambert_per_sample(orc, fp32):
    """FP64: exact to 1e-9.  The float32 instantiation (the kernel's
    precision contract: compensated float optical depth, FP64 tau* and
    remainder) to float rounding of the interaction distance t (~99.6 here,
    a camera far away: a few ulp(t) = 2^-23 t each) and of the shadow ray."""
    tol = 2e-6 if fp32 else 1e-9
    vol, lights, cam = _setup()
    spp, seed = 512, 3
    cs = orc.camera_samples(vol, lights, G, cam, spp, 0.5, seed, fp32=fp32)
    sbar = SIGMA
    words = orc.philox_stream(seed, orc.TAG_CAMERA, 0, 1, 1)  # shape check only
    assert words.shape == (1, 1, 4)
    d = -cs["wo"]
    n_ok = 0
    for py in range(cam.height):
        for px in range(cam.width):
            for k in range(spp):
                w = orc.philox(seed, [py * cam.width + px, 0, (1 << 24) | k, 0])
                u3 = orc.uniform(w)[3]
                o = np.array(cam.eye)
                dd = d[py, px, k]
                t0 = (1.0 - o[2]) / dd[2]
                t1 = (0.0 - o[2]) / dd[2]
                tau_star = -math.log(1 - u3)
                if cs["valid"][py, px, k]:
                    x = cs["x"][py, px, k]
                    t = np.dot(x - o, dd)
                    t_tol = 4 * SIGMA * t * 2.0 ** -23 if fp32 else 0.0
                    assert abs(SIGMA * (t - t0) - tau_star) < tol * max(1, tau_star) + t_tol
                    # shadow ray straight up to z = 1: T = exp(-sigma (1 - z))
                    p = (1 - G * G) / (1 + G * G - 2 * G * np.dot(dd, [0, 0, 1])) ** 1.5 / (4 * math.pi)
                    want = p * math.exp(-SIGMA * (1.0 - x[2]))
                    assert abs(cs["Ld"][py, px, k, 0] - want) < 1e-12 + tol * want
                    n_ok += 1
                else:
                    assert tau_star >= SIGMA * (t1 - t0) * (1 - tol) - (4 * SIGMA * t1 * 2.0 ** -23 if fp32 else 0.0)
    assert n_ok > spp


@pytest.mark.parametrize("mode", ["march", "march32", "delta64", "delta32"])
def test_single_scatter_closed_form(orc, mode):
    vol, lights, cam = _setup()
    spp = 8192
    step = 0.5 if mode.startswith("march") else 0.0
    cs = orc.camera_samples(vol, lights, G, cam, spp, step, seed=5, fp32=mode.endswith("32"))
    contrib = (cs["albedo"] * cs["Ld"])[..., 0]
    m, se = _mean_se(contrib)
    assert abs(m - _closed_form()) < 5 * se


@pytest.mark.parametrize("fp32", [False, True])
def test_one_bounce_path_tracer_equals_tracking_renderer(orc, fp32):
    vol, lights, cam = _setup(4, 3)
    spp = 256
    pt = orc.path_trace(vol, lights, G, cam, spp, max_bounces=1, seed=9, fp32=fp32)
    nr = orc.render_neural(vol, lights, G, cam, spp, 0.0, seed=9, fp32=fp32)
    assert np.allclose(pt, nr, rtol=1e-5 if fp32 else 1e-12, atol=1e-12)
    m = pt.mean()
    assert abs(m - _closed_form()) < 0.05 * _closed_form()


def test_photon_map_indirect_matches_path_tracer(orc):
    """Physics pin of Algorithm 1 + the radiance estimate + Compose: in a
    homogeneous box, direct light by NEE plus photon-map indirect light at
    the first interaction reproduces the multi-bounce path tracer."""
    from oracle import field
    A, sigma, g = 0.85, 3.0, 0.5
    vol = I.Volume(np.ones((8, 8, 8), np.float32), sigma, A, I.tf_constant(1.0))
    lights = [I.Light(I.DIRECTIONAL, tuple(np.array([0.3, 0.4, 1.0]) / np.linalg.norm([0.3, 0.4, 1.0])), (1.0, 1.0, 1.0))]
    cam = I.Camera((2.2, 1.4, 1.9), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 30.0, 6, 6)
    res = 8
    tr = orc.trace_photons(vol, lights, (g,), 1 << 19, 16, res, seed=21, use_rr=True, fp32=False)
    cache = orc.build_cache(tr)
    csig = orc.cell_sigma(vol, res)
    spp = 1024
    cs = orc.camera_samples(vol, lights, g, cam, spp, 0.0, seed=4, fp32=False)
    vm = cs["valid"]
    q = field.query_from_sample(cs["x"][vm], cs["wo"][vm], g)
    q[:, 5] = np.float32(g)
    Li = np.zeros_like(cs["Ld"])
    Li[vm] = orc.estimate_targets(q, (g,), cache, csig)
    neural = (cs["albedo"] * (cs["Ld"] + Li)).sum(2) / spp
    pt = orc.path_trace(vol, lights, g, cam, 4096, 16, seed=8, fp32=False)
    direct = (cs["albedo"] * cs["Ld"]).sum(2) / spp
    indirect_n = neural.mean() - direct.mean()
    indirect_pt = pt.mean() - direct.mean()
    assert indirect_pt > 0.2 * pt.mean()            # multiple scattering matters here
    assert abs(indirect_n - indirect_pt) < 0.06 * indirect_pt
    # the field target stands for the in-scattered radiance itself: dropping
    # the 1/sigma normalisation or the phase function would miss by far more
    assert abs(neural.mean() - pt.mean()) < 0.04 * pt.mean()


def test_pooled_primary_grid_samples_the_same_free_flight(orc):
    """Camera rays tracked over the brick grid max-pooled to 16-voxel bricks
    (brick_primary) sample the same free-flight distribution as over the
    4-voxel brick grid: per-pixel scatter fractions and mean scatter depths
    agree within their sampling error, on a heterogeneous volume."""
    import dataclasses
    sc = I.scene_judge(40, 3, 3, 1)
    base = dataclasses.replace(sc.volume, brick=4)
    pooled = dataclasses.replace(sc.volume, brick=4, brick_primary=16)
    spp = 6000
    a = orc.camera_samples(base, sc.lights, 0.0, sc.camera, spp, 0.0, seed=31)
    b = orc.camera_samples(pooled, sc.lights, 0.0, sc.camera, spp, 0.0, seed=32)
    pa, pb = a["valid"].mean(axis=2), b["valid"].mean(axis=2)
    se = np.sqrt(pa * (1 - pa) / spp + pb * (1 - pb) / spp) + 1e-12
    assert np.all(np.abs(pa - pb) < 5 * se), (pa, pb)
    eye = np.array(sc.camera.eye)
    for y in range(3):
        for x in range(3):
            da = np.linalg.norm(a["x"][y, x][a["valid"][y, x]] - eye, axis=1)
            db = np.linalg.norm(b["x"][y, x][b["valid"][y, x]] - eye, axis=1)
            if da.size > 50 and db.size > 50:
                s = np.sqrt(da.var() / da.size + db.var() / db.size)
                assert abs(da.mean() - db.mean()) < 5 * s + 1e-9
    assert pa.mean() > 0.05
