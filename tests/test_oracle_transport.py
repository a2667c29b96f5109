"""Pins of the oracle's photon tracing (Algorithm 1) and cache (Sec. 3.3).

  * delta tracking samples free-flight distances from Exp(sigma_t) truncated
    at the box (Kolmogorov-Smirnov), with null collisions against a larger
    majorant; over the brick-majorant grid in a heterogeneous volume the
    distances follow 1 - exp(-int sigma) (optical depth by quadrature) and
    ratio tracking's mean is exp(-int sigma); brick majorants bound sigma_t;
  * directional emission covers the box's projection: the fraction of
    photons entering the unit cube is (|vx|+|vy|+|vz|)/3;
  * point emission is isotropic: the fraction entering the cube is its solid
    angle / 4 pi (Van Oosterom-Strackee triangle formula);
  * energy bookkeeping: emitted = escaped + absorbed + truncated + RR, and
    nothing is absorbed at albedo 1;
  * stored powers: the record at interaction j carries P_emit * A^(j-1), the
    power arriving there (before this vertex's albedo);
  * keys decode to the photon's light and phase, and the cache equals the
    per-key sum of record powers.
"""
import math

import numpy as np
import pytest
from scipy import stats

from paper_2304_07338_b300 import inputs as I


def _homog(n=4, alpha=1.0, rgb=(1, 1, 1), ss=1.0, albedo=1.0, tf=None):
    return I.Volume(np.ones((n, n, n), np.float32), ss, albedo,
                    I.tf_constant(alpha, rgb) if tf is None else tf)


def test_delta_tracking_free_flight_distribution(orc):
    # alpha = 0.4 at the volume's density but the table peaks at 1.0, so the
    # majorant is 2.5x sigma_t and 60% of tentative collisions are null
    tf = np.array([[1, 1, 1, 1.0], [1, 1, 1, 0.4]], np.float32)
    vol = I.Volume(np.ones((4, 4, 4), np.float32), 3.0, 1.0, tf)
    sigma = 3.0 * 0.4
    d, steps = orc.free_flight(vol, [0.5, 0.5, -1.0], [0.0, 0.0, 1.0], 100000, seed=11)
    esc = d < 0
    p_esc = math.exp(-sigma)
    assert abs(esc.mean() - p_esc) < 5 * math.sqrt(p_esc * (1 - p_esc) / d.size)
    t = d[~esc]
    cdf = lambda s: (1 - np.exp(-sigma * s)) / (1 - p_esc)
    assert stats.kstest(t, cdf).pvalue > 1e-3
    assert steps / d.size > sigma            # tentative collisions per unit length ~ majorant


def _optical_depth(orc, vol, o, d, s_max, n=20001):
    s = np.linspace(0.0, s_max, n)
    pts = np.asarray(o)[None, :] + s[:, None] * np.asarray(d)[None, :]
    sig = vol.sigma_scale * np.interp(orc.density(vol, pts), np.linspace(0, 1, vol.tf.shape[0]), vol.tf[:, 3])
    tau = np.concatenate([[0.0], np.cumsum(0.5 * (sig[1:] + sig[:-1]) * np.diff(s))])
    return s, tau


@pytest.mark.parametrize("n,B", [(48, 8), (48, 16), (44, 16), (37, 4)])
def test_brick_majorants_bound_sigma(orc, n, B):
    import dataclasses
    vol = dataclasses.replace(I.scene_judge(n).volume, brick=B)
    nb = -(-n // B)
    for fp32 in (False, True):
        m = orc.brick_majorants(vol, fp32)
        assert m.shape == (nb, nb, nb)
        rng = np.random.default_rng(4)
        p = rng.uniform(0, 1, (50000, 3))
        sig = vol.sigma_scale * orc.density(vol, p, fp32)        # alpha = density for this TF
        b = np.minimum((p * n / B).astype(int), nb - 1)
        assert np.all(sig <= m[b[:, 2], b[:, 1], b[:, 0]])
    # tight: the mean brick majorant is below the global one (well below for small bricks)
    assert m.mean() < (0.9 if B <= 8 else 0.99) * orc.majorant(vol)


@pytest.mark.parametrize("B", [8, 16, 4])
def test_grid_delta_tracking_in_heterogeneous_volume(orc, B):
    import dataclasses
    vol = dataclasses.replace(I.scene_judge(40).volume, brick=B)
    o, d = np.array([0.3, 0.62, -0.5]), np.array([0.15, -0.05, 1.0])
    d = d / np.linalg.norm(d)
    t0 = (0.0 - o[2]) / d[2]
    t1 = (1.0 - o[2]) / d[2]
    s, tau = _optical_depth(orc, vol, o + t0 * d, d, t1 - t0)
    dist, _ = orc.free_flight(vol, o, d, 60000, seed=21)
    esc = dist < 0
    p_esc = math.exp(-tau[-1])
    assert abs(esc.mean() - p_esc) < 5 * math.sqrt(p_esc * (1 - p_esc) / dist.size) + 2e-3
    cdf = lambda x: (1 - np.exp(-np.interp(x, s, tau))) / (1 - p_esc)
    assert stats.kstest(dist[~esc], cdf).pvalue > 1e-3
    mean, var = orc.ratio_mean(vol, o + t0 * d, d, t1 - t0, 60000, seed=22)
    assert abs(mean - p_esc) < 5 * math.sqrt(var / 60000) + 2e-3


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("v", [(0.0, 0.0, 1.0), (1.0, 1.0, 0.5), (-0.3, 0.8, -0.2)])
def test_directional_emission_covers_projection(orc, v, fp32):
    vol = _homog(alpha=1.0, ss=1e4, albedo=0.0)
    u = np.array(v) / np.linalg.norm(v)
    light = I.Light(I.DIRECTIONAL, tuple(u), (1.0, 1.0, 1.0))
    N = 100000
    tr = orc.trace_photons(vol, [light], (0.0,), N, max_bounces=2, res=4, seed=3, use_rr=False, fp32=fp32)
    frac = tr["tally"][2, 0] / tr["tally"][0, 0]          # absorbed at the first hit
    want = np.abs(u).sum() / 3.0
    assert abs(frac - want) < 5 * math.sqrt(want * (1 - want) / N) + 1e-6


def _solid_angle_cube(p):
    def tri(a, b, c):
        a, b, c = a - p, b - p, c - p
        la, lb, lc = np.linalg.norm(a), np.linalg.norm(b), np.linalg.norm(c)
        num = abs(np.dot(a, np.cross(b, c)))
        den = la * lb * lc + np.dot(a, b) * lc + np.dot(a, c) * lb + np.dot(b, c) * la
        return 2 * math.atan2(num, den)
    total = 0.0
    for ax in range(3):
        for side in (0.0, 1.0):
            normal_out = -1.0 if side == 0.0 else 1.0
            if (p[ax] - side) * normal_out <= 0:
                continue                         # face not visible
            o = [a for a in range(3) if a != ax]
            corners = []
            for (s, t) in [(0, 0), (1, 0), (1, 1), (0, 1)]:
                c = np.zeros(3); c[ax] = side; c[o[0]] = s; c[o[1]] = t
                corners.append(c)
            total += tri(corners[0], corners[1], corners[2]) + tri(corners[0], corners[2], corners[3])
    return total


@pytest.mark.parametrize("fp32", [False, True])
def test_point_emission_isotropic(orc, fp32):
    vol = _homog(alpha=1.0, ss=1e4, albedo=0.0)
    lights = I.point_lights(2, seed=4)
    N = 100000
    for li, L in enumerate(lights):
        t1 = orc.trace_photons(vol, [L], (0.0,), N, max_bounces=2, res=4, seed=5 + li, use_rr=False, fp32=fp32)
        frac = t1["tally"][2, 0] / t1["tally"][0, 0]
        want = _solid_angle_cube(np.array(L.v)) / (4 * math.pi)
        assert abs(frac - want) < 5 * math.sqrt(want * (1 - want) / N) + 1e-6


@pytest.mark.parametrize("fp32", [False, True])
def test_energy_balance(orc, fp32):
    sc = I.scene_judge(32)
    tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, 3000, 16, 16, seed=7, fp32=fp32)
    t = tr["tally"]
    assert np.allclose(t[0], t[1:].sum(0), rtol=1e-12, atol=0)
    assert t[3].sum() >= 0 and t[2].min() > 0


def test_albedo_one_absorbs_nothing(orc):
    vol = _homog(alpha=1.0, ss=8.0, albedo=1.0)
    tr = orc.trace_photons(vol, I.point_lights(1, 2), (0.0, 0.5), 5000, 16, 8, seed=1, use_rr=False, fp32=False)
    t = tr["tally"]
    assert np.all(t[2] == 0.0) and np.all(t[4] == 0.0)
    assert np.allclose(t[1] + t[3], t[0], rtol=1e-13)


def test_record_power_is_arriving_power(orc):
    A = 0.7
    vol = _homog(alpha=1.0, ss=6.0, albedo=A)
    lights = [I.Light(I.DIRECTIONAL, (0.0, 0.0, 1.0), (1.0, 2.0, 0.5))]
    N = 4000
    tr = orc.trace_photons(vol, lights, (-0.5,), N, 16, 8, seed=2, use_rr=False, fp32=False)
    pe = np.array([1.0, 2.0, 0.5]) * 3.0 / N
    S = tr["keys"].shape[1]
    j = np.arange(S) + 2
    want = pe[None, None, :] * (A ** (j - 1))[None, :, None]
    mask = np.arange(S)[None, :] < tr["nrec"][:, None]
    assert mask.sum() > 1000
    assert np.allclose(tr["phis"][mask], np.broadcast_to(want, tr["phis"].shape)[mask], rtol=1e-6)


def test_keys_and_cache_invariants(orc):
    sc = I.scene_judge(32)
    N, res = 2000, 16
    tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, N, 16, res, seed=9)
    rec = orc.flatten_records(tr)
    ng = len(sc.g_set)
    lg = rec["key"] // res ** 3
    assert np.all(lg == (rec["pid"] // (ng * N)) * ng + (rec["pid"] // N) % ng)
    assert np.all(rec["slot"] < 15)
    cache = orc.build_cache(tr)
    assert cache["counts"].sum() == rec["key"].size
    sums = np.zeros((tr["n_keys"], 3))
    np.add.at(sums, rec["key"].astype(np.int64), rec["phi"].astype(np.float64))
    assert np.allclose(cache["cache64"], sums, rtol=1e-14, atol=0)
    ks = np.repeat(np.arange(tr["n_keys"]), cache["counts"])
    assert np.array_equal(ks, cache["key"].astype(np.int64))


def test_fp32_and_fp64_tracers_agree_statistically(orc):
    sc = I.scene_judge(32)
    a = orc.trace_photons(sc.volume, sc.lights, sc.g_set, 20000, 16, 8, seed=1, fp32=True)
    b = orc.trace_photons(sc.volume, sc.lights, sc.g_set, 20000, 16, 8, seed=2, fp32=False)
    na, nb = a["nrec"].sum(), b["nrec"].sum()
    assert abs(na - nb) < 5 * math.sqrt(na + nb) + 0.02 * na
    assert abs(a["tally"][1, 0] - b["tally"][1, 0]) / a["tally"][0, 0] < 0.02


@pytest.mark.parametrize("B,Bs", [(4, 16), (8, 32), (4, 64)])
def test_thinned_ratio_tracking(orc, B, Bs):
    """Shadow rays walking the grid pooled to Bs-voxel bricks and thinning
    its tentative collisions to the B-voxel brick majorants: the mean is
    exp(-tau) by quadrature, and the variance is that of plain ratio
    tracking with the B-voxel majorants (it is the same estimator).  An
    optically moderate ray (tau ~ 1.5) keeps the variance estimates sharp."""
    import dataclasses
    vol = dataclasses.replace(I.scene_judge(40).volume, brick=B, sigma_scale=3.0)
    thin = dataclasses.replace(vol, brick_shadow=Bs)
    o, d = np.array([0.3, 0.62, -0.5]), np.array([0.15, -0.05, 1.0])
    d = d / np.linalg.norm(d)
    t0, t1 = (0.0 - o[2]) / d[2], (1.0 - o[2]) / d[2]
    s, tau = _optical_depth(orc, vol, o + t0 * d, d, t1 - t0)
    assert 0.5 < tau[-1] < 3.0
    n = 100000
    m_t, v_t = orc.ratio_mean(thin, o + t0 * d, d, t1 - t0, n, seed=41)
    m_p, v_p = orc.ratio_mean(vol, o + t0 * d, d, t1 - t0, n, seed=42)
    want = math.exp(-tau[-1])
    assert abs(m_t - want) < 5 * math.sqrt(v_t / n) + 1e-4 * want
    assert abs(m_p - want) < 5 * math.sqrt(v_p / n) + 1e-4 * want
    assert 0.9 < v_t / v_p < 1.1
