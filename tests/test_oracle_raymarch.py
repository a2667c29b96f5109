"""Pins of the oracle's ray-marching renderer with the field at every step
(Sec. 3.6: the field replaces the multiple-scattering term in ray marching).

Homogeneous box (sigma, albedo A), directional light along +z, camera far
above looking down -z (near-orthographic):
  * segment weights telescope: with the light off and a field whose weights
    are all zero (L' = 0, so L_i = 10^0 = 1 everywhere) every pixel is
    A (1 - exp(-sigma)) exactly, whatever the step and the jitter;
  * direct light: per sample, with the march offset u read from the camera
    stream, the sum over segments of exp(-sigma s0) (1 - exp(-sigma len))
    A p_g(-1) E exp(-sigma (s0 + u len)) (Beer-Lambert along both rays);
    averaged over u it is the closed form sum of
    A p E exp(-2 sigma s0) (1 - exp(-sigma len))^2 / (sigma len), which tends
    to the single-scattering integral A p E (1 - exp(-2 sigma)) / 2 at second
    order in the step;
  * every field query sits on the ray at its segment's sample point with the
    outgoing direction -d (theta' = 0 here) and the render's g.
"""
import math

import numpy as np
import pytest

from oracle import field as F
from paper_2304_07338_b300 import inputs as I

SIGMA, ALB, G = 1.5, 0.8, 0.5


def _setup(W=2, H=2, E=1.0):
    vol = I.Volume(np.ones((8, 8, 8), np.float32), SIGMA, ALB, I.tf_constant(1.0))
    light = I.Light(I.DIRECTIONAL, (0.0, 0.0, 1.0), (E, E, E))
    cam = I.Camera((0.5, 0.5, 100.0), (0.5, 0.5, 0.5), (0.0, 1.0, 0.0), 0.01, W, H)
    return vol, [light], cam


def _p_back():
    return (1 - G * G) / (1 + G) ** 3 / (4 * math.pi)      # p_g(mu = -1)


@pytest.mark.parametrize("step", [0.5, 1.7])
def test_weights_telescope_with_constant_field(orc, step):
    vol, lights, cam = _setup(E=0.0)
    desc = F.FieldDesc(2, 32, 1, F.PREC_F32, 5.0, 0)
    w = np.zeros(desc.n_params())
    img, parts = orc.render_raymarched(vol, lights, G, cam, 3, step, 7, weights=w, desc=desc, return_parts=True)
    # rays leave the vertical by < 1e-4 rad: path length 1 to within 1e-8
    np.testing.assert_allclose(img, ALB * (1 - math.exp(-SIGMA)), rtol=1e-7)
    assert np.all(parts["direct"] == 0)
    # queries: on the ray, direction theta' = 0 (straight up), phase g
    q = parts["q"]
    assert np.all(np.abs(q[:, 3]) < 1e-3) and np.all(q[:, 5] == G)
    # one query per segment: ceil(length / h), the length exceeding 1 by ~1e-9
    # (a sliver segment may follow the last full one)
    nseg = math.ceil(1.0 / (step / 8))
    assert np.all((parts["count"] == nseg) | (parts["count"] == nseg + 1))


def test_direct_light_per_sample_beer_lambert(orc):
    vol, lights, cam = _setup()
    step, spp, seed = 0.5, 16, 11
    img, parts = orc.render_raymarched(vol, lights, G, cam, spp, step, seed, return_parts=True)
    h = step / 8
    D = parts["direct"].reshape(cam.height, cam.width, spp, 3)
    for py in range(cam.height):
        for px in range(cam.width):
            for k in range(spp):
                u = orc.uniform(orc.philox(seed, [py * cam.width + px, 0, (1 << 24) | k, 0]))
                # the ray: entry depth 0 at z = 1, length ~ 1 (near-orthographic)
                o = np.array(cam.eye)
                jx, jy = u[0], u[1]
                # exact ray length through the slab 0 <= z <= 1 from its direction
                th = math.tan(0.5 * 0.01 * math.pi / 180)
                a = (2 * (px + jx) / cam.width - 1) * th * cam.width / cam.height
                b = (1 - 2 * (py + jy) / cam.height) * th
                d = np.array([a, b, -1.0])          # f = -z, r = +x... direction up to orientation
                d /= np.linalg.norm(d)
                length = 1.0 / abs(d[2])
                n = math.ceil(length / h)
                s0 = np.arange(n) * h
                ln = np.minimum(s0 + h, length) - s0
                zdepth = (s0 + u[2] * ln) * abs(d[2])            # depth below z = 1
                want = np.sum(np.exp(-SIGMA * s0) * -np.expm1(-SIGMA * ln) * ALB * _p_back() *
                              np.exp(-SIGMA * zdepth))
                assert abs(D[py, px, k, 0] - want) < 1e-6 * want, (D[py, px, k, 0], want)


def test_direct_light_converges_to_single_scattering(orc):
    vol, lights, cam = _setup()
    closed = ALB * _p_back() * (1 - math.exp(-2 * SIGMA)) / 2
    errs = []
    for step in (2.0, 1.0, 0.5, 0.25):
        h = step / 8
        n = math.ceil(1 / h)
        s0 = np.arange(n) * h
        ln = np.minimum(s0 + h, 1.0) - s0
        expect = np.sum(ALB * _p_back() * np.exp(-2 * SIGMA * s0) * np.expm1(-SIGMA * ln) ** 2 / (SIGMA * ln))
        img = orc.render_raymarched(vol, lights, G, cam, 512, step, 3)
        m = img[..., 0].mean()
        se = img[..., 0].std() / math.sqrt(img[..., 0].size)
        # the sample mean is the jitter average (a few standard errors; the
        # per-pixel values vary only through u)
        assert abs(m - expect) < 4 * max(se, 1e-12) + 1e-4 * expect, (step, m, expect)
        errs.append(abs(expect - closed) / closed)
    # the jitter-averaged quadrature converges to the integral at second order
    assert errs[-1] < 1e-3 and errs[0] > errs[1] > errs[2] > errs[3]
    assert 3.2 < errs[2] / errs[3] < 4.8
