"""Pins of the oracle's training-sample generator and radiance estimate
(Sec. 3.3): queries are uniform over occupied cells, positions uniform inside
their cell, directions uniform on the sphere and g uniform over G; the grid
cell radiance estimate equals the hand-computed sum for a one-record cache
and is linear in the records."""
import math

import numpy as np
import pytest

from paper_2304_07338_b300 import inputs as I


def test_query_sampler_distribution(orc):
    res = 4
    occ = np.array([1, 5, 6, 30, 63])
    G = (-0.5, 0.0, 0.5)
    B = 60000
    q, gi = orc.sample_queries(occ, res, G, B, step=3, seed=11)
    cell = (np.floor(q[:, 0] * res) + res * (np.floor(q[:, 1] * res) + res * np.floor(q[:, 2] * res))).astype(int)
    # every query sits in an occupied cell, which are all equally likely
    assert set(np.unique(cell)) <= set(occ.tolist())
    cnt = np.array([(cell == c).sum() for c in occ])
    assert np.abs(cnt - B / len(occ)).max() < 5 * math.sqrt(B / len(occ))
    # direction uniform on the sphere
    w = orc.query_direction(q)
    assert np.allclose(np.linalg.norm(w, axis=1), 1.0)
    assert np.abs(w.mean(0)).max() < 5 / math.sqrt(3 * B)
    assert abs((w[:, 2] ** 2).mean() - 1 / 3) < 0.01
    assert np.all((q[:, 3] >= 0) & (q[:, 3] <= 1) & (q[:, 4] >= 0) & (q[:, 4] < 1))
    gcnt = np.bincount(gi, minlength=3)
    assert np.abs(gcnt - B / 3).max() < 5 * math.sqrt(B / 3)
    assert np.array_equal(q[:, 5], np.asarray(G, np.float32)[gi].astype(np.float64))
    # the draws depend on the step
    q2, _ = orc.sample_queries(occ, res, G, B, step=4, seed=11)
    assert not np.allclose(q, q2)


def test_estimate_single_record(orc):
    res, G = 2, (0.0, 0.5)
    n_keys = 1 * len(G) * res ** 3
    # one record in cell 3 for (light 0, g index 1)
    key = 1 * res ** 3 + 3
    counts = np.zeros(n_keys, np.int64); counts[key] = 1
    offsets = np.concatenate([[0], np.cumsum(counts)])
    d = np.array([[0.0, 0.6, 0.8]], np.float32)
    phi = np.array([[0.2, 0.4, 0.1]], np.float32)
    cache = dict(offsets=offsets, dir=d, phi=phi, res=res, n_lights=1, n_g=2)
    csig = np.full(res ** 3, 2.5)
    # cell 3 = (1, 1, 0): x in [0.5,1) x [0.5,1) x [0,0.5)
    q = np.array([[0.75, 0.6, 0.2, 0.3, 0.1, 0.5], [0.75, 0.6, 0.2, 0.3, 0.1, 0.0], [0.1, 0.1, 0.1, 0.3, 0.1, 0.5]])
    L = orc.estimate_targets(q, G, cache, csig)
    w = orc.query_direction(q[:1])[0]
    mu = float(np.dot(d[0].astype(np.float64), w))
    p = (1 - 0.25) / (1 + 0.25 - 2 * 0.5 * mu) ** 1.5 / (4 * math.pi)
    want = p * phi[0].astype(np.float64) / ((1 / res ** 3) * 2.5)
    assert np.allclose(L[0], want, rtol=1e-12)
    assert np.all(L[1] == 0) and np.all(L[2] == 0)     # other phase / other cell


def test_estimate_is_linear_in_records(orc):
    sc = I.scene_judge(32)
    res = 8
    tr = orc.trace_photons(sc.volume, sc.lights, sc.g_set, 4000, 16, res, seed=3)
    cache = orc.build_cache(tr)
    csig = orc.cell_sigma(sc.volume, res)
    occ = orc.occupied_cells(cache, csig)
    q, _ = orc.sample_queries(occ, res, sc.g_set, 500, 0, 1)
    L = orc.estimate_targets(q, sc.g_set, cache, csig)
    half = dict(cache)
    half["phi"] = cache["phi"] * np.float32(0.5)
    assert np.allclose(orc.estimate_targets(q, sc.g_set, half, csig), 0.5 * L, rtol=1e-12)
    assert np.all(L >= 0) and L.max() > 0


def test_cell_sigma_is_mean_of_fine_voxels(orc):
    rng = np.random.default_rng(0)
    data = rng.uniform(0, 1, (8, 8, 8)).astype(np.float32)
    vol = I.Volume(data, 3.0, 1.0, I.tf_linear_gray())
    cs = orc.cell_sigma(vol, 4)
    want = 3.0 * data.astype(np.float64).reshape(4, 2, 4, 2, 4, 2).mean(axis=(1, 3, 5)).reshape(-1)
    assert np.allclose(cs, want, rtol=1e-14)
