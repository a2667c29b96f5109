"""Pins of the oracle's phase function and volume access.

Henyey-Greenstein (Sec. 3.2, Fig. hg_plot): unit normalisation over the
sphere, mean cosine equal to g, the isotropic value 1/(4 pi) at g = 0, and a
sampler whose cosine follows the pdf (chi-square) and reproduces the inverse
CDF exactly.  Volume: trilinear interpolation reproduces voxel values at voxel
centres and linear fields exactly, is zero outside [0,1]^3; the majorant
bounds every sigma_t.
"""
import math

import numpy as np
import pytest
from scipy import integrate

from paper_2304_07338_b300 import inputs as I


@pytest.mark.parametrize("g", [-0.9, -0.5, 0.0, 0.3, 0.75, 0.9])
def test_hg_normalised_and_mean_cosine(orc, g):
    f = lambda mu: orc.lib().orc_hg_eval(g, mu)
    norm = 2 * math.pi * integrate.quad(f, -1, 1, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
    mean = 2 * math.pi * integrate.quad(lambda mu: mu * f(mu), -1, 1, epsabs=1e-13, epsrel=1e-13, limit=200)[0]
    assert abs(norm - 1.0) < 1e-10
    assert abs(mean - g) < 1e-10


def test_hg_isotropic_value(orc):
    assert abs(orc.hg_eval(0.0, [-1, 0, 0.3, 1]) - 1 / (4 * math.pi)).max() < 1e-15
    # forward scattering: g > 0 favours mu = +1 (incoming and outgoing travel
    # directions aligned)
    assert orc.hg_eval(0.75, [1.0])[0] > orc.hg_eval(0.75, [-1.0])[0]


def _hg_cdf(g, mu):
    if abs(g) < 1e-12:
        return (mu + 1) / 2
    return (1 - g * g) / (2 * g) * (1 / np.sqrt(1 + g * g - 2 * g * mu) - 1 / (1 + g))


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("g", [-0.75, 0.0, 0.5, 0.75])
def test_hg_sampler_distribution(orc, g, fp32):
    n = 200000
    xi = orc.uniform(orc.philox_stream(9, 2, 0, n // 2, 1).reshape(-1)).reshape(-1, 2)
    d = np.array([0.36, -0.48, 0.8])
    out = orc.hg_sample(g, d, xi, fp32=fp32)
    assert np.allclose(np.linalg.norm(out, axis=1), 1.0, atol=1e-6 if fp32 else 1e-13)
    mu = out @ d
    if abs(g) >= 1e-3:
        gg = g * g
        want = (1 + gg - ((1 - gg) / (1 - g + 2 * g * xi[:, 0])) ** 2) / (2 * g)
    else:
        want = 1 - 2 * xi[:, 0]
    assert np.max(np.abs(mu - np.clip(want, -1, 1))) < (2e-5 if fp32 else 1e-12)
    edges = np.linspace(-1, 1, 41)
    h = np.histogram(mu, edges)[0]
    p = np.diff(_hg_cdf(g, edges))
    e = p * mu.size
    m = e > 5
    chi2 = ((h[m] - e[m]) ** 2 / e[m]).sum()
    dof = m.sum() - 1
    assert chi2 < dof + 6 * math.sqrt(2 * dof)
    perp = out - mu[:, None] * d[None, :]          # azimuth uniform about d
    assert np.abs(perp.mean(0)).max() < 5 * math.sqrt(0.5 / mu.size) + 1e-3


def _vol(data, tf=None, ss=1.0, alb=1.0):
    return I.Volume(data, ss, alb, I.tf_linear_gray() if tf is None else tf)


@pytest.mark.parametrize("fp32", [False, True])
def test_density_at_voxel_centres(orc, fp32):
    rng = np.random.default_rng(3)
    data = rng.uniform(0, 1, (5, 6, 7)).astype(np.float32)
    v = _vol(data)
    k, j, i = np.meshgrid(np.arange(5), np.arange(6), np.arange(7), indexing="ij")
    pts = np.stack([(i + 0.5) / 7, (j + 0.5) / 6, (k + 0.5) / 5], -1).reshape(-1, 3)
    got = orc.density(v, pts, fp32)
    assert np.allclose(got, data.reshape(-1), atol=1e-6 if fp32 else 1e-14)


def test_density_reproduces_linear_field_and_zero_outside(orc):
    n = 8
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    data = (0.1 + 0.2 * x + 0.3 * y + 0.25 * z).astype(np.float64)
    v = _vol(data.astype(np.float32))
    rng = np.random.default_rng(0)
    p = rng.uniform(0.5 / n, 1 - 0.5 / n, (1000, 3))
    want = 0.1 + 0.2 * p[:, 0] + 0.3 * p[:, 1] + 0.25 * p[:, 2]
    assert np.allclose(orc.density(v, p), want, atol=1e-6)
    out = np.array([[-1e-9, 0.5, 0.5], [0.5, 1.0 + 1e-9, 0.5], [0.5, 0.5, 2.0]])
    assert np.all(orc.density(v, out) == 0.0)
    q = np.array([[0.5 / n * 0.3, 0.5, 0.5]])          # clamp to edge
    q2 = np.array([[0.5 / n, 0.5, 0.5]])
    assert abs(orc.density(v, q)[0] - orc.density(v, q2)[0]) < 1e-12


def test_density_u8_and_f16_decoding(orc):
    data8 = np.array([[[0, 51], [102, 255]], [[17, 34], [68, 200]]], np.uint8)
    v = _vol(data8)
    k, j, i = np.meshgrid(np.arange(2), np.arange(2), np.arange(2), indexing="ij")
    pts = np.stack([(i + 0.5) / 2, (j + 0.5) / 2, (k + 0.5) / 2], -1).reshape(-1, 3)
    assert np.allclose(orc.density(v, pts), data8.reshape(-1) / 255.0, atol=1e-15)
    data16 = np.array([0.0, 0.25, 1.0, 0.1, 0.7, 0.33, 0.999, 0.5], np.float16).reshape(2, 2, 2)
    v = _vol(data16)
    assert np.allclose(orc.density(v, pts), data16.reshape(-1).astype(np.float64), atol=0)


@pytest.mark.parametrize("fp32", [False, True])
def test_majorant_bounds_sigma(orc, fp32):
    sc = I.scene_small(16)
    vol = sc.volume
    sbar = orc.majorant(vol, fp32)
    rng = np.random.default_rng(2)
    p = rng.uniform(0, 1, (20000, 3))
    sig = vol.sigma_scale * orc.density(vol, p, fp32)      # linear grey TF: alpha = density
    assert sig.max() <= sbar
    assert sbar <= vol.sigma_scale * float(vol.data.max()) * 1.001
    # peaked transfer function: the majorant takes the table's interior maximum
    tf = np.array([[1, 1, 1, 0.0], [1, 1, 1, 1.0], [1, 1, 1, 0.2]], np.float32)
    v2 = I.Volume(np.full((4, 4, 4), 0.9, np.float32), 3.0, 1.0, tf)
    assert abs(orc.majorant(v2) - 3.0 * 1.0009765625) < 1e-12
