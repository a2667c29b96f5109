"""Pins of the oracle's multiresolution hash-grid encoding (Sec. 3.4).

The encoding interpolates a per-level table multilinearly between the
vertices of the cell holding the point.  Fixed from outside the oracle:
  * affine reproduction: a dense level whose table holds an affine function
    of the vertex coordinates returns that function of the point exactly
    (multilinear interpolation reproduces affine functions), which fixes the
    dense index order, the corner weights and the level offsets; the same on
    a hashed level for tables written only at the corners' own slots when
    those do not collide;
  * weights: non-negative, summing to one; at a vertex, one corner has
    weight one;
  * continuity across cell faces;
  * the field's gradient with respect to MLP weights and table entries
    against central differences in FP64 (the field is linear in the tables);
  * initialisation bounds and the parameter layout.
"""
import math

import numpy as np
import pytest

from oracle import field as F


def _desc(**kw):
    base = dict(hidden=32, n_hidden=2, encoding=F.ENC_HASHGRID, hash_levels=4, hash_features=2,
                hash_log2_size=10, hash_base_res=4, hash_scale=2.0, seed=5)
    base.update(kw)
    return F.FieldDesc(**base)


def test_layout_and_init():
    d = _desc()
    w = F.init_weights(d)
    assert w.size == d.n_params()
    assert d.n_in == 2 * 4 * 2 + 1
    offs = d.table_offsets()
    assert offs[0][0] >= d.n_mlp() and offs[0][0] % 8 == 0
    prev = 0
    for j, g in enumerate(d.grids()):
        for l in range(g.levels):
            assert offs[j][l] % 8 == 0 and offs[j][l] >= prev
            n = g.entries(l) * g.features
            t = w[offs[j][l]:offs[j][l] + n]
            assert np.all(np.abs(t) <= 1e-4) and np.std(t) > 3e-5
            assert np.all(w[offs[j][l] + n:offs[j][l] + g.level_floats(l)] == 0)
            prev = offs[j][l] + g.level_floats(l)
            # dense iff the vertices fit the table
            assert g.dense(l) == ((g.res(l) + 1) ** g.dim <= 2 ** g.log2_size)
    for (o, i), W in zip(d.shapes(), F.unflatten(w, d)):
        assert np.all(np.abs(W) <= math.sqrt(6.0 / i))


@pytest.mark.parametrize("dim", [3, 2])
def test_weights_partition_of_unity_and_vertices(dim):
    g = F.HashGrid(dim, 3, 1, 12, 5, 1.5)
    rng = np.random.default_rng(1)
    x = rng.random((500, dim))
    for l in range(g.levels):
        idx, wgt = F.hash_corners(g, l, x)
        assert np.all(wgt >= 0) and np.allclose(wgt.sum(1), 1.0, atol=1e-12)
        N = g.res(l)
        # points exactly on vertices (N = 5, 7, 11 are not powers of two, so
        # pick vertex coordinates whose ratio is exact in float32: v / N * N)
        v = rng.integers(0, N + 1, (50, dim))
        xv = (v / N).astype(np.float32).astype(np.float64)
        ok = np.all(np.float32(xv) * np.float32(N) == v.astype(np.float32), axis=1)
        idx, wgt = F.hash_corners(g, l, xv[ok])
        assert np.all(np.isclose(wgt.max(1), 1.0))


@pytest.mark.parametrize("dim", [3, 2])
def test_dense_level_reproduces_affine(dim):
    g = F.HashGrid(dim, 3, 2, 16, 3, 2.0)            # 4, 7, 13 cells per axis: all dense
    rng = np.random.default_rng(2)
    a = rng.normal(size=(2, dim))
    b = rng.normal(size=2)
    x = rng.random((400, dim))
    for l in range(g.levels):
        assert g.dense(l)
        N = g.res(l)
        # vertex v at linear index sum_k v_k (N+1)^k holds a . v / N + b
        lin = np.arange(g.entries(l))
        v = np.stack([(lin // (N + 1) ** k) % (N + 1) for k in range(dim)], 1)
        tab = v @ a.T / N + b
        idx, wgt = F.hash_corners(g, l, x)
        feat = np.einsum("bc,bcf->bf", wgt, tab[idx])
        # the cell is taken in float32 (p = float32(x) N): compare with the
        # affine function at that point
        p = np.float32(x.astype(np.float32)) * np.float32(N)
        want = p.astype(np.float64) @ a.T / N + b
        np.testing.assert_allclose(feat, want, rtol=0, atol=1e-12)


def test_hashed_level_reproduces_affine_without_collisions():
    g = F.HashGrid(3, 6, 1, 14, 4, 2.0)              # levels 4.. are hashed (T = 16384)
    rng = np.random.default_rng(3)
    a = rng.normal(size=3)
    for l in range(g.levels):
        if g.dense(l):
            continue
        N = g.res(l)
        for x in rng.random((200, 3)):
            idx, wgt = F.hash_corners(g, l, x[None])
            if len(set(idx[0])) < 8:
                continue                              # corners collide: not an affine test
            p = np.float32(x.astype(np.float32)) * np.float32(N)
            i = np.minimum(np.floor(p), N - 1)
            tab = np.zeros(g.entries(l))
            for c in range(8):
                v = i + np.array([(c >> k) & 1 for k in range(3)])
                tab[idx[0, c]] = a @ v / N
            feat = wgt[0] @ tab[idx[0]]
            assert abs(feat - a @ p.astype(np.float64) / N) < 1e-12


def test_continuity_across_faces():
    d = _desc(hash_features=4)
    w = F.init_weights(d)
    rng = np.random.default_rng(4)
    q = rng.random((64, 6))
    N = d.grids()[0].res(2)
    face = (np.floor(q[:, 0] * N) + 1) / N
    lo, hi = q.copy(), q.copy()
    lo[:, 0] = np.nextafter(face.astype(np.float32), np.float32(0)).astype(np.float64)
    hi[:, 0] = np.nextafter(face.astype(np.float32), np.float32(2)).astype(np.float64)
    ok = hi[:, 0] < 1
    hl, _ = F.hash_encode(w, lo[ok], d)
    hh, _ = F.hash_encode(w, hi[ok], d)
    assert np.abs(hl - hh).max() < 1e-9


def _loss(w, q, y, d):
    yhat, cache = F.forward(w, q, d)
    l, dy = F.rel_mse(yhat, y)
    return l, cache, dy


@pytest.mark.parametrize("levels,features", [(3, 2), (2, 8)])
def test_gradient_matches_central_differences(levels, features):
    d = _desc(hash_levels=levels, hash_features=features, hash_base_res=3)
    w = F.init_weights(d).astype(np.float64)
    # larger tables so that the encoding moves the loss measurably
    rng = np.random.default_rng(5)
    w[d.n_mlp():] = rng.normal(size=w.size - d.n_mlp()) * 0.5
    q = rng.random((24, 6))
    y = rng.random((24, 3))
    l0, cache, dy = _loss(w, q, y, d)
    g = F.backward(w, cache, dy, d)
    assert g.size == d.n_params()
    # touched table entries and a few MLP weights
    touched = np.nonzero(g[d.n_mlp():])[0] + d.n_mlp()
    assert touched.size > 0
    pick = np.concatenate([rng.choice(touched, 20, replace=False), rng.choice(d.n_mlp(), 10, replace=False)])
    h = 1e-6
    for i in pick:
        wp, wm = w.copy(), w.copy()
        wp[i] += h
        wm[i] -= h
        fd = (_loss(wp, q, y, d)[0] - _loss(wm, q, y, d)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)) + 1e-9, (i, fd, g[i])
    # untouched table entries get no gradient
    untouched = np.setdiff1d(np.arange(d.n_mlp(), d.n_params()), touched)
    assert np.all(g[untouched] == 0)


def test_g_passes_through_raw():
    d = _desc()
    w = F.init_weights(d)
    q = np.random.default_rng(6).random((10, 6))
    h, _ = F.hash_encode(w, q, d)
    assert h.shape == (10, d.n_in)
    np.testing.assert_array_equal(h[:, -1], q[:, 5])
