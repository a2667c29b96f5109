"""CPU oracle for the Photon Field Networks hot path (arXiv 2304.07338).

TEST INFRASTRUCTURE ONLY: imported by tests/, by the smoke check and by the
benchmark's CPU-baseline leg, never by the product path.  It shares no code
with the CUDA library.  Tracing and gathering run in pf_oracle.cpp (FP64, plus
a float32 instantiation for the FP-decided integer work); the field network,
its gradients, the loss, Adam and the log target codec are plain numpy FP64
(field.py).  Each function names the passage of the paper it follows.

Parity pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import math
from typing import Dict, Optional, Sequence

import numpy as np

from . import build as _build
from . import field  # noqa: F401  (re-export)

_lib = None

TAG_CAMERA, TAG_PHOTON, TAG_QUERY, TAG_INIT = 1, 2, 3, 4


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        _declare(_lib)
    return _lib


def _declare(L):
    P = C.c_void_p
    i32, i64, u32, u64, f64 = C.c_int, C.c_int64, C.c_uint32, C.c_uint64, C.c_double
    L.orc_philox.argtypes = [u64, P, P]
    L.orc_philox_stream.argtypes = [u64, u32, u32, i64, i32, P]
    L.orc_philox_item.argtypes = [u64, u32, u32, u64, i64, P]
    L.orc_lnf.argtypes = [P, P, i64]
    L.orc_sincos2pif.argtypes = [P, P, P, i64]
    L.orc_atan2f.argtypes = [P, P, P, i64]
    L.orc_encode_f32.argtypes = [P, i64, i32, P]
    L.orc_query_f32.argtypes = [P, P, C.c_float, i64, P]
    L.orc_hg_eval.argtypes = [f64, f64]
    L.orc_hg_eval.restype = f64
    L.orc_hg_sample.argtypes = [f64, P, P, i64, P, i32]
    L.orc_density.argtypes = [i32, i32, i32, i32, P, P, i64, P, i32]
    L.orc_majorant.argtypes = [i32, i32, i32, i32, P, f64, f64, P, i32, i32]
    L.orc_majorant.restype = f64
    L.orc_free_flight.argtypes = [i32, i32, i32, i32, P, f64, P, i32, i32, P, P, i64, u64, P, P]
    L.orc_brick_majorants.argtypes = [i32, i32, i32, i32, P, f64, P, i32, i32, i32, P]
    L.orc_ratio_mean.argtypes = [i32, i32, i32, i32, P, f64, P, i32, i32, i32, P, P, f64, i64, u64, P]
    L.orc_ratio_mean.restype = f64
    L.orc_trace_photons.argtypes = [i32, i32, i32, i32, P, f64, f64, P, i32, i32,
                                    P, P, P, i32, P, i32, u64, i32, i32, u64, i32, i32, u64, u64,
                                    P, P, P, P, P, P]
    L.orc_camera_samples.argtypes = [i32, i32, i32, i32, P, f64, f64, P, i32, i32, i32, i32,
                                     P, P, P, i32, f64, P, P, P, f64, i32, i32,
                                     i32, f64, u64, i32, i32, i32, i32, i32, P, P, P, P, P]
    L.orc_path_trace.argtypes = [i32, i32, i32, i32, P, f64, f64, P, i32, i32,
                                 P, P, P, i32, f64, P, P, P, f64, i32, i32,
                                 i32, i32, u64, i32, i32, i32, i32, P, i64, P]
    L.orc_cell_sigma.argtypes = [i32, i32, i32, i32, P, f64, P, i32, i32, P]
    L.orc_estimate.argtypes = [P, P, P, i64, P, P, P, P, P, i32, i32, i32, P]
    L.orc_raymarch.argtypes = [i32, i32, i32, i32, P, f64, f64, P, i32, P, P, P, i32, f64, P, P, P, f64, i32, i32,
                               i32, f64, u64, i32, i32, P, P, P, P, P]
    L.orc_estimate_knn.argtypes = [P, P, P, i64, P, P, P, P, P, i64, i32, C.c_float, P, P, i32, P, P, P]


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


# ------------------------------------------------------------------ scene marshalling
class _Vol:
    """Keeps the arrays alive while the C side reads them."""

    def __init__(self, vol):
        data = np.ascontiguousarray(vol.data)
        if data.dtype == np.float16:
            data = data.view(np.uint16)
        self.data = data
        self.tf = np.ascontiguousarray(vol.tf, np.float32)
        nz, ny, nx = vol.data.shape
        code = {np.dtype(np.float32): 0, np.dtype(np.float16): 1, np.dtype(np.uint8): 2}[np.dtype(vol.data.dtype)]
        self.args = (nx, ny, nz, code, _p(self.data))
        self.ss = float(vol.sigma_scale)
        self.alb = float(vol.albedo)
        self.tfargs = (_p(self.tf), int(self.tf.shape[0]))
        self.brick = int(getattr(vol, "brick", 8))
        self.brick_primary = int(getattr(vol, "brick_primary", 0))
        self.brick_shadow = int(getattr(vol, "brick_shadow", 0))


class _Lights:
    def __init__(self, lights):
        self.kind = np.array([l.kind for l in lights], np.int32)
        self.v = np.array([l.v for l in lights], np.float64).reshape(-1)
        self.rgb = np.array([l.rgb for l in lights], np.float64).reshape(-1)
        self.n = len(lights)
        self.args = (_p(self.kind), _p(self.v), _p(self.rgb), self.n)


class _Cam:
    """Camera parameters as the C ABI carries them (float32), widened to FP64."""

    def __init__(self, cam):
        f32 = lambda v: np.array(v, np.float32).astype(np.float64)
        self.eye, self.at, self.up = f32(cam.eye), f32(cam.at), f32(cam.up)
        self.args = (_p(self.eye), _p(self.at), _p(self.up), float(np.float32(cam.fovy_deg)), int(cam.width),
                     int(cam.height))


# ------------------------------------------------------------------ random numbers
def philox(seed: int, ctr: Sequence[int]) -> np.ndarray:
    """One Philox4x32-10 block (Salmon et al., SC'11)."""
    c = np.array(ctr, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().orc_philox(seed, _p(c), _p(out))
    return out


def philox_stream(seed: int, tag: int, sub: int, n_items: int, n_blocks: int) -> np.ndarray:
    """Raw words [item][block][4] of the stream (seed, tag, sub)."""
    out = np.zeros((n_items, n_blocks, 4), np.uint32)
    lib().orc_philox_stream(seed, tag, sub, n_items, n_blocks, _p(out))
    return out


def philox_item(seed: int, tag: int, sub: int, item: int, n_blocks: int) -> np.ndarray:
    """Raw words [block][4] of one item of the stream (seed, tag, sub)."""
    out = np.zeros((n_blocks, 4), np.uint32)
    lib().orc_philox_item(seed, tag, sub, item, n_blocks, _p(out))
    return out


def uniform(words: np.ndarray) -> np.ndarray:
    """u = (x >> 8) * 2^-24 in [0, 1)."""
    return (words >> np.uint32(8)).astype(np.float64) * (1.0 / 16777216.0)


def lnf(x: np.ndarray) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float32)
    y = np.zeros_like(x)
    lib().orc_lnf(_p(x), _p(y), x.size)
    return y


def sincos2pif(u: np.ndarray):
    u = np.ascontiguousarray(u, np.float32)
    s, c = np.zeros_like(u), np.zeros_like(u)
    lib().orc_sincos2pif(_p(u), _p(s), _p(c), u.size)
    return s, c


def atan2f(y: np.ndarray, x: np.ndarray) -> np.ndarray:
    """The project's own float32 atan2 (half-angle step + Taylor series)."""
    y = np.ascontiguousarray(y, np.float32)
    x = np.ascontiguousarray(x, np.float32)
    out = np.zeros_like(y)
    lib().orc_atan2f(_p(y), _p(x), _p(out), y.size)
    return out


def encode_f32(q: np.ndarray, n_freq: int) -> np.ndarray:
    """The frequency encoding in the float32 steps of the tensor-core fields
    (own turn-based sine / cosine at k = 0, 4, 8, ..., double-angle formulas
    in between); (B, 12 n_freq) as float64 (exact)."""
    q = np.ascontiguousarray(np.asarray(q).reshape(-1, 6), np.float32)
    out = np.zeros((q.shape[0], 12 * n_freq), np.float32)
    lib().orc_encode_f32(_p(q), q.shape[0], int(n_freq), _p(out))
    return out.astype(np.float64)


def query_f32(x: np.ndarray, wo: np.ndarray, g: float) -> np.ndarray:
    """Field queries (x, theta', phi', g) formed in float32 from float32
    interaction points and outgoing directions, as the renderer forms them
    (Sec. 3.1's normalised spherical coordinates with the own atan2);
    returned as float64 (exact)."""
    x = np.ascontiguousarray(np.asarray(x).reshape(-1, 3), np.float32)
    wo = np.ascontiguousarray(np.asarray(wo).reshape(-1, 3), np.float32)
    q = np.zeros((x.shape[0], 6), np.float32)
    lib().orc_query_f32(_p(x), _p(wo), float(np.float32(g)), x.shape[0], _p(q))
    return q.astype(np.float64)


# ------------------------------------------------------------------ phase function
def hg_eval(g: float, mu) -> np.ndarray:
    """Henyey-Greenstein phase function (Sec. 3.2, Fig. hg_plot)."""
    mu = np.atleast_1d(np.asarray(mu, np.float64))
    return np.array([lib().orc_hg_eval(float(g), float(m)) for m in mu])


def hg_sample(g: float, d, xi: np.ndarray, fp32: bool = False) -> np.ndarray:
    d = np.ascontiguousarray(d, np.float64)
    xi = np.ascontiguousarray(xi, np.float64).reshape(-1, 2)
    out = np.zeros((xi.shape[0], 3))
    lib().orc_hg_sample(float(g), _p(d), _p(xi), xi.shape[0], _p(out), int(fp32))
    return out


# ------------------------------------------------------------------ volume
def density(vol, pts: np.ndarray, fp32: bool = False) -> np.ndarray:
    v = _Vol(vol)
    pts = np.ascontiguousarray(pts, np.float64).reshape(-1, 3)
    out = np.zeros(pts.shape[0])
    lib().orc_density(*v.args, _p(pts), pts.shape[0], _p(out), int(fp32))
    return out


def majorant(vol, fp32: bool = False) -> float:
    v = _Vol(vol)
    return lib().orc_majorant(*v.args, v.ss, v.alb, *v.tfargs, int(fp32))


def brick_majorants(vol, fp32: bool = False) -> np.ndarray:
    """Majorant per brick (x fastest), bounding sigma_t inside each brick."""
    v = _Vol(vol)
    nz, ny, nx = vol.data.shape
    g = [(a + v.brick - 1) // v.brick for a in (nx, ny, nz)]
    out = np.zeros(g[0] * g[1] * g[2])
    lib().orc_brick_majorants(*v.args, v.ss, *v.tfargs, v.brick, int(fp32), _p(out))
    return out.reshape(g[2], g[1], g[0])


def ratio_mean(vol, o, d, t_end: float, n: int, seed: int):
    """Mean and variance of n ratio-tracking transmittance estimates (walking
    the grid pooled to vol.brick_shadow and thinned to vol.brick, if set)."""
    v = _Vol(vol)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    var = np.zeros(1)
    m = lib().orc_ratio_mean(*v.args, v.ss, *v.tfargs, v.brick, v.brick_shadow, _p(o), _p(d), float(t_end), n, seed,
                             _p(var))
    return m, float(var[0])


def free_flight(vol, o, d, n: int, seed: int):
    """n delta-tracking free-flight distances from o along d (-1 = escaped)."""
    v = _Vol(vol)
    o = np.ascontiguousarray(o, np.float64)
    d = np.ascontiguousarray(d, np.float64)
    out = np.zeros(n)
    steps = np.zeros(1, np.int64)
    lib().orc_free_flight(*v.args, v.ss, *v.tfargs, v.brick, _p(o), _p(d), n, seed, _p(out), _p(steps))
    return out, int(steps[0])


# ------------------------------------------------------------------ photon tracing (Algorithm 1)
def trace_photons(vol, lights, g_set, n_per, max_bounces: int = 16, res: int = 64, seed: int = 1,
                  use_rr: bool = True, fp32: bool = True, p_begin: int = 0, p_end: Optional[int] = None) -> Dict:
    """Multi-phase photon tracing (Algorithm 1) into per-photon record slots."""
    v, L = _Vol(vol), _Lights(lights)
    g = np.ascontiguousarray(g_set, np.float32)
    total = L.n * len(g) * n_per
    if p_end is None:
        p_end = total
    P = p_end - p_begin
    S = max(max_bounces - 1, 1)
    keys = np.full((P, S), 0xFFFFFFFF, np.uint32)
    dirs = np.zeros((P, S, 3), np.float32)
    phis = np.zeros((P, S, 3), np.float32)
    poss = np.zeros((P, S, 3), np.float32)
    nrec = np.zeros(P, np.int32)
    tally = np.zeros(15)
    lib().orc_trace_photons(*v.args, v.ss, v.alb, *v.tfargs, v.brick, *L.args, _p(g), len(g), n_per, max_bounces, res,
                            seed, int(use_rr), int(fp32), p_begin, p_end,
                            _p(keys), _p(dirs), _p(phis), _p(poss), _p(nrec), _p(tally))
    return dict(keys=keys, dirs=dirs, phis=phis, poss=poss, nrec=nrec, tally=tally.reshape(5, 3),
                n_keys=L.n * len(g) * res ** 3, res=res, n_lights=L.n, n_g=len(g), p_begin=p_begin)


def flatten_records(tr: Dict):
    """Records in (photon id, bounce) order: key, photon id, slot, dir, power,
    position."""
    S = tr["keys"].shape[1]
    mask = np.arange(S)[None, :] < tr["nrec"][:, None]
    pid = np.broadcast_to((np.arange(tr["keys"].shape[0]) + tr["p_begin"])[:, None], mask.shape)[mask]
    slot = np.broadcast_to(np.arange(S)[None, :], mask.shape)[mask]
    return dict(key=tr["keys"][mask], pid=pid.astype(np.int64), slot=slot.astype(np.int64),
                dir=tr["dirs"][mask], phi=tr["phis"][mask], pos=tr["poss"][mask])


def build_cache(tr: Dict) -> Dict:
    """Binning and cache: counts per key, CSR offsets, records grouped by key
    (stable, so photon/bounce order is kept inside a key) and the per-key
    power sums in FP64 rounded to float32."""
    rec = flatten_records(tr)
    n_keys = tr["n_keys"]
    counts = np.bincount(rec["key"].astype(np.int64), minlength=n_keys).astype(np.int64)
    offsets = np.zeros(n_keys + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    order = np.argsort(rec["key"], kind="stable")
    cache64 = np.zeros((n_keys, 3))
    np.add.at(cache64, rec["key"].astype(np.int64), rec["phi"].astype(np.float64))
    rid = ((rec["pid"] << 4) | rec["slot"]).astype(np.uint32)
    return dict(counts=counts, offsets=offsets, dir=rec["dir"][order], phi=rec["phi"][order],
                key=rec["key"][order], pos=rec["pos"][order], rid=rid[order],
                phase=((rec["key"][order].astype(np.int64) // tr["res"] ** 3) % tr["n_g"]).astype(np.int32), cache=cache64.astype(np.float32), cache64=cache64,
                res=tr["res"], n_lights=tr["n_lights"], n_g=tr["n_g"])


def cell_sigma(vol, res: int) -> np.ndarray:
    """Mean sigma_t over the fine voxel centres inside each cache cell."""
    v = _Vol(vol)
    out = np.zeros(res ** 3)
    lib().orc_cell_sigma(*v.args, v.ss, *v.tfargs, res, _p(out))
    return out


def occupied_cells(cache: Dict, csig: np.ndarray) -> np.ndarray:
    """Cells (ascending) with records for some light and phase and sigma > 0."""
    nc = cache["res"] ** 3
    tot = cache["counts"].reshape(-1, nc).sum(0)
    return np.nonzero((tot > 0) & (csig > 0))[0].astype(np.int64)


# ------------------------------------------------------------------ training samples (Sec. 3.3)
def sample_queries(occ: np.ndarray, res: int, g_set, B: int, step: int, seed: int):
    """Training queries: cell uniform over the occupied list, position uniform
    in the cell, direction uniform on the sphere, g uniform over G.
    Returns (q (B,6) float64, g index (B,))."""
    w = philox_stream(seed, TAG_QUERY, step, B, 2).astype(np.uint64)
    r24 = w >> np.uint64(8)
    M = np.uint64(len(occ))
    cell = occ[((r24[:, 0, 0] * M) >> np.uint64(24)).astype(np.int64)]
    cx, cy, cz = cell % res, (cell // res) % res, cell // (res * res)
    u = r24.astype(np.float64) * (1.0 / 16777216.0)
    x = (cx + u[:, 0, 1]) / res
    y = (cy + u[:, 0, 2]) / res
    z = (cz + u[:, 0, 3]) / res
    wz = 1.0 - 2.0 * u[:, 1, 0]
    theta = np.arccos(np.clip(wz, -1.0, 1.0)) / math.pi
    phi = u[:, 1, 1]
    gi = ((r24[:, 1, 2] * np.uint64(len(g_set))) >> np.uint64(24)).astype(np.int64)
    g = np.asarray(g_set, np.float32).astype(np.float64)[gi]
    return np.stack([x, y, z, theta, phi, g], 1), gi


def query_direction(q: np.ndarray) -> np.ndarray:
    """Outgoing direction from the query's normalised spherical coordinates."""
    th = math.pi * q[:, 3]
    ph = 2.0 * math.pi * q[:, 4]
    return np.stack([np.sin(th) * np.cos(ph), np.sin(th) * np.sin(ph), np.cos(th)], 1)


def estimate_targets(q: np.ndarray, g_set, cache: Dict, csig: np.ndarray) -> np.ndarray:
    """Radiance estimate per query (Sec. 3.3.1, Eq. of the KNN estimator, with
    the cache cell as the gather region): sum over lights and over the records
    of the query's phase in its cell of p_g(dir . w) Phi / (V_cell sigma_cell)."""
    q = np.ascontiguousarray(q, np.float64)
    gs = np.asarray(g_set, np.float32)
    gi = np.array([int(np.nonzero(gs == np.float32(v))[0][0]) for v in q[:, 5]], np.int32)
    x = np.ascontiguousarray(q[:, :3])
    w = np.ascontiguousarray(query_direction(q))
    off = np.ascontiguousarray(cache["offsets"], np.int64)
    rdir = np.ascontiguousarray(cache["dir"], np.float32)
    rphi = np.ascontiguousarray(cache["phi"], np.float32)
    cs = np.ascontiguousarray(csig, np.float64)
    out = np.zeros((q.shape[0], 3))
    lib().orc_estimate(_p(x), _p(w), _p(gi), q.shape[0], _p(off), _p(rdir), _p(rphi), _p(cs), _p(gs),
                       len(gs), cache["n_lights"], cache["res"], _p(out))
    return out


def estimate_targets_knn(q: np.ndarray, g_set, cache: Dict, csig: np.ndarray, K: int, r_max: float):
    """Phase-selective KNN radiance estimate per query (Sec. 3.3.1, the
    adaptive-radius estimator over the K nearest photons of the query's phase,
    search radius capped at r_max; box units).  `cache` needs the records'
    pos, rid, phase, dir and phi (build_cache, or any dict with those
    arrays).  Returns (L_s (B,3) float64, k used (B,), radius r (B,) float32)."""
    q = np.ascontiguousarray(q, np.float64)
    gs = np.asarray(g_set, np.float32)
    gi = np.array([int(np.nonzero(gs == np.float32(v))[0][0]) for v in q[:, 5]], np.int32)
    x = np.ascontiguousarray(q[:, :3], np.float32)
    w = np.ascontiguousarray(query_direction(q))
    pos = np.ascontiguousarray(cache["pos"], np.float32)
    rid = np.ascontiguousarray(cache["rid"], np.uint32)
    ph = np.ascontiguousarray(cache["phase"], np.int32)
    rdir = np.ascontiguousarray(cache["dir"], np.float32)
    rphi = np.ascontiguousarray(cache["phi"], np.float32)
    cs = np.ascontiguousarray(csig, np.float64)
    res = round(cs.size ** (1.0 / 3.0))
    assert res ** 3 == cs.size
    B = q.shape[0]
    out = np.zeros((B, 3))
    k = np.zeros(B, np.int32)
    r = np.zeros(B, np.float32)
    lib().orc_estimate_knn(_p(x), _p(w), _p(gi), B, _p(pos), _p(rid), _p(ph), _p(rdir), _p(rphi), pos.shape[0],
                           int(K), float(np.float32(r_max)), _p(cs), _p(gs), res, _p(out), _p(k), _p(r))
    return out, k, r


# ------------------------------------------------------------------ rendering (Algorithm 2)
def camera_samples(vol, lights, g: float, cam, spp: int, step_vox: float, seed: int,
                   fp32: bool = False, rows=None, cols=None) -> Dict:
    """RayGeneration + VolumeSampling + DirectIllumination per camera sample
    (pixels in rows [y0, y1) and columns [x0, x1))."""
    v, L, cm = _Vol(vol), _Lights(lights), _Cam(cam)
    y0, y1 = rows if rows is not None else (0, cam.height)
    x0, x1 = cols if cols is not None else (0, cam.width)
    n = (y1 - y0) * (x1 - x0) * spp
    valid = np.zeros(n, np.uint8)
    x, wo, alb, Ld = (np.zeros((n, 3)) for _ in range(4))
    lib().orc_camera_samples(*v.args, v.ss, v.alb, *v.tfargs, v.brick, v.brick_primary, v.brick_shadow, *L.args, float(g), *cm.args, spp,
                             float(step_vox), seed, int(fp32), y0, y1, x0, x1,
                             _p(valid), _p(x), _p(wo), _p(alb), _p(Ld))
    shp = (y1 - y0, x1 - x0, spp)
    return dict(valid=valid.reshape(shp).astype(bool), x=x.reshape(shp + (3,)), wo=wo.reshape(shp + (3,)),
                albedo=alb.reshape(shp + (3,)), Ld=Ld.reshape(shp + (3,)))


def render_neural(vol, lights, g: float, cam, spp: int, step_vox: float, seed: int,
                  weights=None, desc=None, scales=None, fp32: bool = False, rows=None, cols=None,
                  return_parts: bool = False):
    """Neural path tracing (Algorithm 2): camera samples, field prediction and
    exponential decode at the valid samples, then Compose
    L = 1/spp sum_k albedo_k (L_d,k + L_i,k) with unit MIS weights."""
    cs = camera_samples(vol, lights, g, cam, spp, step_vox, seed, fp32, rows, cols)
    Li = np.zeros_like(cs["Ld"])
    if weights is not None:
        vm = cs["valid"]
        # float32 instantiation: the queries as the renderer forms them in
        # float32; FP64: the exact spherical coordinates
        qv = query_f32(cs["x"][vm], cs["wo"][vm], g) if fp32 else field.query_from_sample(cs["x"][vm], cs["wo"][vm], g)
        y, _ = field.forward(weights, qv, desc, scales)
        Li[vm] = field.log_decode(y, desc.psi)
    img = (cs["albedo"] * (cs["Ld"] + Li)).sum(axis=2) / spp
    if return_parts:
        return img, cs, Li
    return img


def render_raymarched(vol, lights, g: float, cam, spp: int, step_vox: float, seed: int,
                      weights=None, desc=None, scales=None, rows=None, return_parts: bool = False):
    """Ray marching with the photon field at every step (Sec. 3.6): per
    camera sample the sum over the march segments of a_s albedo_s (L_d + L_i)
    (see orc_raymarch), averaged over the samples of a pixel; L_i from the
    field (weights, desc, scales as for render_neural), or 0 without one.
    Returns the image of rows [y0, y1) (and the per-ray direct part, query
    counts, queries and weights with return_parts)."""
    v, L, cm = _Vol(vol), _Lights(lights), _Cam(cam)
    y0, y1 = rows if rows is not None else (0, cam.height)
    n = (y1 - y0) * cam.width * spp
    D = np.zeros((n, 3))
    cnt = np.zeros(n, np.int64)
    args = (*v.args, v.ss, v.alb, *v.tfargs, *L.args, float(g), *cm.args, spp, float(step_vox), seed, y0, y1)
    lib().orc_raymarch(*args, _p(D), _p(cnt), None, None, None)
    rad = D.copy()
    q = w = None
    if weights is not None:
        off = np.zeros(n + 1, np.int64)
        np.cumsum(cnt, out=off[1:])
        q = np.zeros((int(off[-1]), 6))
        w = np.zeros((int(off[-1]), 3))
        D2 = np.zeros((n, 3))
        cnt2 = np.zeros(n, np.int64)
        lib().orc_raymarch(*args, _p(D2), _p(cnt2), _p(off), _p(q), _p(w))
        ray = np.repeat(np.arange(n), cnt)
        for a in range(0, q.shape[0], 1 << 18):
            y, _ = field.forward(weights, q[a:a + (1 << 18)], desc, scales)
            np.add.at(rad, ray[a:a + (1 << 18)], field.log_decode(y, desc.psi) * w[a:a + (1 << 18)])
    img = rad.reshape(y1 - y0, cam.width, spp, 3).mean(2)
    if return_parts:
        return img, dict(direct=D, count=cnt, q=q, w=w)
    return img


def path_trace(vol, lights, g: float, cam, spp: int, max_bounces: int = 16, seed: int = 1,
               use_rr: bool = True, fp32: bool = True, rows=None, pixels: Optional[np.ndarray] = None) -> np.ndarray:
    """Plain multi-bounce path tracer with next-event estimation (Sec. 4,
    baseline); rows [y0, y1) or an explicit (n, 2) list of (x, y) pixels."""
    v, L, cm = _Vol(vol), _Lights(lights), _Cam(cam)
    y0, y1 = rows if rows is not None else (0, cam.height)
    if pixels is not None:
        px = np.ascontiguousarray(pixels, np.int32)
        out = np.zeros((px.shape[0], 3))
        lib().orc_path_trace(*v.args, v.ss, v.alb, *v.tfargs, v.brick, *L.args, float(g), *cm.args, spp, max_bounces,
                             seed, int(use_rr), int(fp32), 0, 0, _p(px), px.shape[0], _p(out))
        return out
    out = np.zeros(((y1 - y0) * cam.width, 3))
    lib().orc_path_trace(*v.args, v.ss, v.alb, *v.tfargs, v.brick, *L.args, float(g), *cm.args, spp, max_bounces,
                         seed, int(use_rr), int(fp32), y0, y1, None, 0, _p(out))
    return out.reshape(y1 - y0, cam.width, 3)


def rmse(a: np.ndarray, b: np.ndarray) -> float:
    """sqrt(mean((a-b)^2)) over all pixels and channels, FP64."""
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return float(math.sqrt(np.mean(d * d)))
