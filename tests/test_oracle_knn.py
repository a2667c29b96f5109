"""Pins of the oracle's phase-selective KNN radiance estimate (Sec. 3.3.1).

The estimate is  L_s = sum_{K nearest photons of phase g} p_g(dir_n . w) Phi_n
/ ((4/3) pi r^3 sigma), with r the K-th distance when the search ball holds at
least K photons and the ball's radius otherwise.  The pins below fix every
part of it from outside the oracle's code:
  * photons on a lattice around the query: the shell counts come from integer
    enumeration, so the selected set, r and the 4/3 pi r^3 volume are known
    in closed form for both the saturated and the radius-limited case;
  * phase selectivity: photons of another phase never count, photons of the
    same phase from any light do;
  * the phase function's orientation: one photon travelling along +z seen
    along +z (forward) or -z (backward) gives (1+g)/(1-g)^2 / 4pi or
    (1-g)/(1+g)^2 / 4pi, closed forms of HG at mu = +1 and -1;
  * Poisson photons of density lambda: the K-nearest estimate K / V_K has
    mean lambda K / (K - 1) (V_K is Gamma(K, lambda)), and the radius-limited
    estimate k / V has mean lambda; an off-by-one in the neighbour index or
    the wrong radius rule moves the mean by 1 / (K - 1).
"""
import math

import numpy as np
import pytest

import oracle as orc

FOUR_PI = 4.0 * math.pi


def _cache(pos, phase, dirs=None, phi=None):
    n = len(pos)
    dirs = np.tile([0.0, 0.0, 1.0], (n, 1)) if dirs is None else dirs
    phi = np.ones((n, 3)) if phi is None else phi
    return dict(pos=np.asarray(pos, np.float32), rid=np.arange(n, dtype=np.uint32),
                phase=np.asarray(phase, np.int32), dir=np.asarray(dirs, np.float32),
                phi=np.asarray(phi, np.float32))


def _query(x, g, w=(0.0, 0.0, 1.0)):
    # normalised spherical coordinates of w (theta' = acos(w_z)/pi, phi' = atan2/2pi mod 1)
    th = math.acos(max(-1.0, min(1.0, w[2]))) / math.pi
    ph = (math.atan2(w[1], w[0]) / (2 * math.pi)) % 1.0
    return np.array([[x[0], x[1], x[2], th, ph, g]])


def _lattice(h, n):
    # points 0.5 + h (i + 1/2), i in [-n, n): the point (0.5, 0.5, 0.5) is a cube centre
    i = np.arange(-n, n)
    I, J, K = np.meshgrid(i, i, i, indexing="ij")
    c = np.stack([I.ravel(), J.ravel(), K.ravel()], 1)
    return 0.5 + h * (c + 0.5), c


def _shell_counts(c):
    # 4 d^2 / h^2 = (2i+1)^2 + (2j+1)^2 + (2k+1)^2, an integer: exact shells
    s = ((2 * c + 1) ** 2).sum(1)
    vals, cnt = np.unique(s, return_counts=True)
    return vals, np.cumsum(cnt)


@pytest.mark.parametrize("K", [8, 32, 56, 100])
def test_lattice_saturated(K):
    h = 1.0 / 64
    pos, c = _lattice(h, 4)
    vals, cum = _shell_counts(c)
    sigma = 2.0
    cache = _cache(pos, np.zeros(len(pos)))
    L, k, r = orc.estimate_targets_knn(_query((0.5, 0.5, 0.5), 0.0), [0.0], cache, np.array([sigma]), K, 0.2)
    # the K-th photon lies on the first shell whose cumulative count reaches K
    shell = vals[np.searchsorted(cum, K)]
    r_want = h * math.sqrt(shell) / 2
    assert k[0] == K
    assert abs(float(r[0]) - r_want) <= 1e-7 * r_want
    want = K / FOUR_PI / (4.0 / 3.0 * math.pi * float(r[0]) ** 3 * sigma)
    np.testing.assert_allclose(L[0], [want] * 3, rtol=1e-12)
    assert abs(want / (K / FOUR_PI / (4.0 / 3.0 * math.pi * r_want ** 3 * sigma)) - 1) < 1e-6


@pytest.mark.parametrize("r2_over_h2", [1.0, 2.0, 5.5])
def test_lattice_radius_limited(r2_over_h2):
    h = 1.0 / 64
    pos, c = _lattice(h, 4)
    vals, cum = _shell_counts(c)
    sigma = 0.5
    r_max = h * math.sqrt(r2_over_h2)
    cache = _cache(pos, np.zeros(len(pos)))
    L, k, r = orc.estimate_targets_knn(_query((0.5, 0.5, 0.5), 0.0), [0.0], cache, np.array([sigma]), 1024, r_max)
    inside = int(cum[np.searchsorted(vals, 4 * r2_over_h2, side="right") - 1])
    assert k[0] == inside
    assert r[0] == np.float32(r_max)
    want = inside / FOUR_PI / (4.0 / 3.0 * math.pi * float(np.float32(r_max)) ** 3 * sigma)
    np.testing.assert_allclose(L[0], [want] * 3, rtol=1e-12)


def test_phase_selective_over_lights():
    h = 1.0 / 64
    pos, _ = _lattice(h, 3)
    base = _cache(pos, np.zeros(len(pos)))
    g_set = [-0.5, 0.0, 0.5]
    q = _query((0.5, 0.5, 0.5), 0.0)
    L0, k0, r0 = orc.estimate_targets_knn(q, g_set, dict(base, phase=np.ones(len(pos), np.int32)), np.array([1.0]),
                                          8, 0.1)
    # phase index 1 is g = 0: the lattice photons count
    assert k0[0] == 8
    # photons of phase 0 and 2 right at the query change nothing
    extra = np.array([[0.5, 0.5, 0.5], [0.5001, 0.5, 0.5]], np.float32)
    mixed = _cache(np.concatenate([pos, extra]), np.concatenate([np.ones(len(pos)), [0, 2]]))
    L1, k1, r1 = orc.estimate_targets_knn(q, g_set, mixed, np.array([1.0]), 8, 0.1)
    assert k1[0] == 8 and r1[0] == r0[0]
    np.testing.assert_array_equal(L1, L0)
    # the same photons labelled phase 1 (another light's photons of this
    # phase), with power 10, are the two nearest: they replace two photons of
    # the first shell, whose distance is still the 8th
    phi = np.concatenate([np.ones((len(pos), 3)), np.full((2, 3), 10.0)])
    same = _cache(np.concatenate([pos, extra]), np.ones(len(pos) + 2), phi=phi)
    L2, k2, r2 = orc.estimate_targets_knn(q, g_set, same, np.array([1.0]), 8, 0.1)
    assert k2[0] == 8 and r2[0] == r0[0]
    want = (6 + 2 * 10) / FOUR_PI / (4.0 / 3.0 * math.pi * float(r0[0]) ** 3)
    np.testing.assert_allclose(L2[0], [want] * 3, rtol=1e-12)


@pytest.mark.parametrize("g", [0.5, -0.3])
def test_phase_function_orientation(g):
    # one photon travelling along +z, 0.01 from the query
    cache = _cache([[0.5, 0.5, 0.51]], [0], phi=[[1.0, 2.0, 3.0]])
    sigma = 3.0
    fwd, k, r = orc.estimate_targets_knn(_query((0.5, 0.5, 0.5), g, (0, 0, 1)), [g], cache, np.array([sigma]), 1, 0.1)
    bwd, _, _ = orc.estimate_targets_knn(_query((0.5, 0.5, 0.5), g, (0, 0, -1)), [g], cache, np.array([sigma]), 1, 0.1)
    assert k[0] == 1
    vol = 4.0 / 3.0 * math.pi * float(r[0]) ** 3
    gg = float(np.float32(g))
    p_fwd = (1 + gg) / (1 - gg) ** 2 / FOUR_PI
    p_bwd = (1 - gg) / (1 + gg) ** 2 / FOUR_PI
    np.testing.assert_allclose(fwd[0], p_fwd * np.array([1.0, 2.0, 3.0]) / (vol * sigma), rtol=1e-9)
    np.testing.assert_allclose(bwd[0], p_bwd * np.array([1.0, 2.0, 3.0]) / (vol * sigma), rtol=1e-9)


def test_empty_and_degenerate():
    cache = _cache([[0.9, 0.9, 0.9]], [0])
    L, k, r = orc.estimate_targets_knn(_query((0.1, 0.1, 0.1), 0.0), [0.0], cache, np.array([1.0]), 16, 0.05)
    assert k[0] == 0 and r[0] == np.float32(0.05) and np.all(L == 0)
    # zero sigma in the query's cell: estimate 0
    L, k, r = orc.estimate_targets_knn(_query((0.9, 0.9, 0.9), 0.0), [0.0], cache, np.zeros(1), 16, 0.05)
    assert k[0] == 1 and np.all(L == 0)


def _poisson(lam, seed):
    rng = np.random.default_rng(seed)
    n = rng.poisson(lam)
    return rng.random((n, 3))


def test_poisson_k_nearest_mean():
    lam, K = 200000, 16
    pos = _poisson(lam, 1)
    cache = _cache(pos, np.zeros(len(pos)))
    rng = np.random.default_rng(2)
    B = 3000
    x = 0.2 + 0.6 * rng.random((B, 3))
    q = np.concatenate([x, np.tile([0.5, 0.25, 0.0], (B, 1))], 1)
    L, k, r = orc.estimate_targets_knn(q, [0.0], cache, np.ones(1), K, 0.15)
    assert np.all(k == K) and np.all(r < 0.15)
    est = L[:, 0] * FOUR_PI                       # = K / V_K
    m, se = est.mean(), est.std() / math.sqrt(B)
    want = lam * K / (K - 1)
    assert abs(m - want) < 4 * se + 0.005 * want, (m, want, se)
    assert abs(m - lam) > 4 * se                  # the K/(K-1) factor is resolved


def test_poisson_radius_limited_mean():
    lam, r_max = 200000, 0.012                    # about 1.45 photons per ball: never saturated at K = 64
    pos = _poisson(lam, 3)
    cache = _cache(pos, np.zeros(len(pos)))
    rng = np.random.default_rng(4)
    B = 4000
    x = 0.1 + 0.8 * rng.random((B, 3))
    q = np.concatenate([x, np.tile([0.5, 0.25, 0.0], (B, 1))], 1)
    L, k, r = orc.estimate_targets_knn(q, [0.0], cache, np.ones(1), 64, r_max)
    assert np.all(k < 64) and np.all(r == np.float32(r_max))
    vol = 4.0 / 3.0 * math.pi * float(np.float32(r_max)) ** 3
    np.testing.assert_allclose(L[:, 0] * FOUR_PI * vol, k, rtol=1e-12)
    m, se = (k / vol).mean(), (k / vol).std() / math.sqrt(B)
    assert abs(m - lam) < 4 * se, (m, lam, se)
