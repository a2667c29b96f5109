"""Python binding of libpf (include/pf.h) with torch tensors as buffers.

Argument marshalling only: every step of the hot path runs in the library's
CUDA kernels.  Tensors supply device pointers; the context's stream is the
torch current stream of its device unless one is given.
"""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence, Tuple

import numpy as np
import torch

from . import _lib
from ._lib import (PfCacheInfo, PfCamera, PfError, PfFieldDesc, PfLight, PfTrainDesc, PfVolume)

PREC = {"f32": 0, "bf16": 1, "f16": 2, "fp8": 3}


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need(t: torch.Tensor, dtype, numel: Optional[int] = None, name: str = "tensor"):
    if not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    if numel is not None and t.numel() < numel:
        raise ValueError("%s has %d elements, need %d" % (name, t.numel(), numel))


class Context:
    """pf_ctx: one device, one stream, the library's scratch."""

    def __init__(self, device: int = 0, stream: Optional[torch.cuda.Stream] = None):
        self.lib = _lib.load()
        self.device = device
        s = stream if stream is not None else torch.cuda.current_stream(device)
        self.stream = s
        h = C.c_void_p()
        st = self.lib.pf_create(C.byref(h), device, C.c_void_p(s.cuda_stream))
        if st != 0:
            raise PfError(st, "pf_create failed")
        self.h = h

    def check(self, st: int):
        if st != 0:
            raise PfError(st, self.lib.pf_last_error(self.h).decode())

    def sync(self):
        self.check(self.lib.pf_sync(self.h))

    def set_counters(self, counters: Optional[torch.Tensor]):
        """Count density lookups into counters[0] (int64 CUDA tensor) or stop (None)."""
        self.check(self.lib.pf_set_counters(self.h, _ptr(counters)))

    STAGES = ("camera", "field", "compose", "path", "train", "photons", "nee")

    def stage_timing(self, enable: bool):
        self.check(self.lib.pf_stage_timing(self.h, int(enable)))

    def stage_times(self):
        """{stage: (milliseconds, launches)} accumulated since the last call."""
        n = len(self.STAGES)
        ms = (C.c_double * n)()
        cnt = (C.c_int * n)()
        self.check(self.lib.pf_stage_times(self.h, ms, cnt, n))
        return {s: (ms[i], cnt[i]) for i, s in enumerate(self.STAGES)}

    def close(self):
        if getattr(self, "h", None):
            self.lib.pf_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Volume:
    """Device-resident volume + transfer function (pf_volume)."""

    def __init__(self, data: torch.Tensor, sigma_scale: float, albedo: float, tf: torch.Tensor,
                 majorant: float = 0.0, brick: int = 8, brick_primary: int = 0, brick_shadow: int = 0):
        code = {torch.float32: 0, torch.float16: 1, torch.uint8: 2}[data.dtype]
        if not data.is_cuda or not data.is_contiguous() or data.dim() != 3:
            raise ValueError("volume data must be a contiguous 3-D CUDA tensor (nz, ny, nx)")
        _need(tf, torch.float32, name="tf")
        self.data, self.tf = data, tf
        nz, ny, nx = data.shape
        self.s = PfVolume(nx, ny, nz, code, data.data_ptr(), float(sigma_scale), float(albedo), tf.data_ptr(),
                          int(tf.shape[0]), float(majorant), None, int(brick), int(brick_primary),
                          int(brick_shadow))
        self.grid = None

    @classmethod
    def from_inputs(cls, vol, device="cuda"):
        """From a paper_2304_07338_b300.inputs.Volume (numpy arrays)."""
        data = torch.from_numpy(np.ascontiguousarray(vol.data)).to(device)
        tf = torch.from_numpy(np.ascontiguousarray(vol.tf, np.float32)).to(device)
        return cls(data, vol.sigma_scale, vol.albedo, tf, brick=getattr(vol, "brick", 8),
                   brick_primary=getattr(vol, "brick_primary", 0), brick_shadow=getattr(vol, "brick_shadow", 0))

    def attach_tiled(self, ctx: Context) -> torch.Tensor:
        """Copy the voxels into 4x4x4 tiles once (same values) and let the
        tracers gather from the copy."""
        nz, ny, nx = self.data.shape
        n = ((nx + 3) // 4) * ((ny + 3) // 4) * ((nz + 3) // 4) * 64
        self.tiled = torch.empty(n, dtype=self.data.dtype, device=self.data.device)
        ctx.check(ctx.lib.pf_volume_tile(ctx.h, C.byref(self.s), _ptr(self.tiled)))
        self.s.tiled_dev = self.tiled.data_ptr()
        return self.tiled

    def brick_majorants(self, ctx: Context) -> torch.Tensor:
        """Brick majorants (computed on the GPU), shape (gz, gy, gx)."""
        nz, ny, nx = self.data.shape
        B = self.s.brick or 8
        g = torch.empty(((nz + B - 1) // B, (ny + B - 1) // B, (nx + B - 1) // B), dtype=torch.float32,
                        device=self.data.device)
        ctx.check(ctx.lib.pf_volume_brick_majorants(ctx.h, C.byref(self.s), _ptr(g)))
        return g

    def attach_brick_majorants(self, ctx: Context) -> torch.Tensor:
        """Compute the brick majorants once and let every call reuse them."""
        self.grid = self.brick_majorants(ctx)
        self.s.brick_majorants_dev = self.grid.data_ptr()
        return self.grid

    def majorant(self, ctx: Context) -> float:
        out = C.c_float()
        ctx.check(ctx.lib.pf_volume_majorant(ctx.h, C.byref(self.s), C.byref(out)))
        return out.value


def _lights(lights) -> tuple:
    arr = (PfLight * len(lights))()
    for i, l in enumerate(lights):
        arr[i].kind = int(l.kind)
        for c in range(3):
            arr[i].v[c] = float(l.v[c])
            arr[i].rgb[c] = float(l.rgb[c])
    return arr, len(lights)


def _camera(cam) -> PfCamera:
    c = PfCamera()
    for i in range(3):
        c.eye[i], c.at[i], c.up[i] = float(cam.eye[i]), float(cam.at[i]), float(cam.up[i])
    c.fovy_deg, c.width, c.height = float(cam.fovy_deg), int(cam.width), int(cam.height)
    return c


class Cache:
    """pf_cache: photon records (CSR by key), per-key counts and power sums."""

    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        info = PfCacheInfo()
        ctx.check(ctx.lib.pf_cache_info(ctx.h, h, C.byref(info)))
        self.info = info

    @property
    def n_records(self):
        return self.info.n_records

    def tally(self) -> np.ndarray:
        return np.array(self.info.tally[:]).reshape(5, 3)

    def export(self):
        i = self.info
        dev = torch.device("cuda", self.ctx.device)
        counts = torch.empty(i.n_keys, dtype=torch.int32, device=dev)
        flux = torch.empty(i.n_keys * 3, dtype=torch.float32, device=dev)
        nr = max(i.n_records, 1)
        key = torch.empty(nr, dtype=torch.int32, device=dev)
        rid = torch.empty(nr, dtype=torch.int32, device=dev)
        rdir = torch.empty(nr * 3, dtype=torch.float32, device=dev)
        rphi = torch.empty(nr * 3, dtype=torch.float32, device=dev)
        rpos = torch.empty(nr * 3, dtype=torch.float32, device=dev)
        occ = torch.empty(max(i.n_occupied, 1), dtype=torch.int32, device=dev)
        csig = torch.empty(i.res ** 3, dtype=torch.float32, device=dev)
        self.ctx.check(self.ctx.lib.pf_cache_export(self.ctx.h, self.h, *map(_ptr, (counts, flux, key, rid, rdir, rphi,
                                                                                     rpos, occ, csig))))
        torch.cuda.synchronize(dev)
        n = i.n_records
        return dict(counts=counts, flux=flux.view(-1, 3), key=key[:n], id=rid[:n], dir=rdir[:3 * n].view(-1, 3),
                    phi=rphi[:3 * n].view(-1, 3), pos=rpos[:3 * n].view(-1, 3), occupied=occ[:i.n_occupied], cell_sigma=csig)

    def sample_queries(self, B: int, step: int, seed: int) -> torch.Tensor:
        q = torch.empty(B * 6, dtype=torch.float32, device=torch.device("cuda", self.ctx.device))
        self.ctx.check(self.ctx.lib.pf_sample_queries(self.ctx.h, self.h, B, step, seed, _ptr(q)))
        return q.view(B, 6)

    def estimate_targets(self, q: torch.Tensor, psi: float = 5.0):
        _need(q, torch.float32, name="q")
        B = q.numel() // 6
        ls = torch.empty(B * 3, dtype=torch.float32, device=q.device)
        lp = torch.empty(B * 3, dtype=torch.float32, device=q.device)
        self.ctx.check(self.ctx.lib.pf_estimate_targets(self.ctx.h, self.h, _ptr(q), B, psi, _ptr(ls), _ptr(lp)))
        return ls.view(B, 3), lp.view(B, 3)

    def estimate_targets_knn(self, q: torch.Tensor, K: int, r_max: float, psi: float = 5.0):
        """Phase-selective K-nearest estimate: (L_s, L', records used, radius)."""
        _need(q, torch.float32, name="q")
        B = q.numel() // 6
        ls = torch.empty(B * 3, dtype=torch.float32, device=q.device)
        lp = torch.empty(B * 3, dtype=torch.float32, device=q.device)
        k = torch.empty(B, dtype=torch.int32, device=q.device)
        r = torch.empty(B, dtype=torch.float32, device=q.device)
        self.ctx.check(self.ctx.lib.pf_estimate_targets_knn(self.ctx.h, self.h, _ptr(q), B, K, r_max, psi, _ptr(ls),
                                                            _ptr(lp), _ptr(k), _ptr(r)))
        return ls.view(B, 3), lp.view(B, 3), k, r

    def free(self):
        if self.h:
            self.ctx.lib.pf_cache_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def build_photon_cache(ctx: Context, vol: Volume, lights, g_set: Sequence[float], photons_per_light_per_g: int,
                       max_bounces: int = 16, cache_res: int = 64, seed: int = 1, use_rr: bool = True) -> Cache:
    la, n = _lights(lights)
    g = (C.c_float * len(g_set))(*[float(x) for x in g_set])
    h = C.c_void_p()
    ctx.check(ctx.lib.pf_build_photon_cache(ctx.h, C.byref(vol.s), la, n, g, len(g_set), int(photons_per_light_per_g),
                                            int(max_bounces), int(cache_res), int(seed), int(use_rr), C.byref(h)))
    return Cache(ctx, h)


class Field:
    """pf_field: photon field network with library-owned weights."""

    def __init__(self, ctx: Context, in_freqs=12, hidden=64, n_hidden=3, prec="f32", psi=5.0, seed=0,
                 encoding: str = "frequency", hash_levels=16, hash_features=8, hash_log2_size=19, hash_base_res=16,
                 hash_scale=2.0):
        """encoding "frequency" (in_freqs per input) or "hashgrid" (the
        hash_* parameters; see pf_field_desc)."""
        self.ctx = ctx
        self.prec = prec
        enc = {"frequency": 0, "hashgrid": 1}[encoding]
        self.desc = PfFieldDesc(int(in_freqs), int(hidden), int(n_hidden), PREC[prec] if isinstance(prec, str) else int(prec),
                                float(psi), int(seed), enc, int(hash_levels), int(hash_features), int(hash_log2_size),
                                int(hash_base_res), float(hash_scale))
        h = C.c_void_p()
        ctx.check(ctx.lib.pf_field_create(ctx.h, C.byref(self.desc), C.byref(h)))
        self.h = h
        self.n_params = ctx.lib.pf_field_num_params(h)

    @property
    def psi(self):
        return self.desc.psi

    def get_weights(self) -> torch.Tensor:
        w = torch.empty(self.n_params, dtype=torch.float32, device=torch.device("cuda", self.ctx.device))
        self.ctx.check(self.ctx.lib.pf_field_get_weights(self.ctx.h, self.h, _ptr(w)))
        return w

    def set_weights(self, w: torch.Tensor):
        _need(w, torch.float32, self.n_params, "weights")
        self.ctx.check(self.ctx.lib.pf_field_set_weights(self.ctx.h, self.h, _ptr(w)))

    def calibrate_fp8(self, q: torch.Tensor):
        _need(q, torch.float32, name="q")
        self.ctx.check(self.ctx.lib.pf_field_calibrate_fp8(self.ctx.h, self.h, _ptr(q), q.numel() // 6))

    def forward(self, q: torch.Tensor, out: Optional[torch.Tensor] = None) -> torch.Tensor:
        _need(q, torch.float32, name="q")
        B = q.numel() // 6
        if out is None:
            out = torch.empty(B, 3, dtype=torch.float32, device=q.device)
        self.ctx.check(self.ctx.lib.pf_field_forward(self.ctx.h, self.h, _ptr(q), B, _ptr(out)))
        return out

    def backward(self, q: torch.Tensor, dy: torch.Tensor) -> torch.Tensor:
        _need(q, torch.float32, name="q")
        _need(dy, torch.float32, name="dy")
        B = q.numel() // 6
        dw = torch.empty(self.n_params, dtype=torch.float32, device=q.device)
        self.ctx.check(self.ctx.lib.pf_field_backward(self.ctx.h, self.h, _ptr(q), _ptr(dy), B, _ptr(dw)))
        return dw

    def loss_gradient(self, q: torch.Tensor, targets: torch.Tensor):
        """(loss, dw): the training loss on targets (L') and its gradient."""
        _need(q, torch.float32, name="q")
        B = q.numel() // 6
        _need(targets, torch.float32, 3 * B, "targets")
        dw = torch.empty(self.n_params, dtype=torch.float32, device=q.device)
        loss = C.c_float()
        self.ctx.check(self.ctx.lib.pf_field_loss_gradient(self.ctx.h, self.h, _ptr(q), _ptr(targets), B, _ptr(dw),
                                                           C.byref(loss)))
        return loss.value, dw

    def adam(self, grad: torch.Tensor, lr: float, beta1=0.9, beta2=0.99, eps=1e-8):
        _need(grad, torch.float32, self.n_params, "grad")
        self.ctx.check(self.ctx.lib.pf_field_adam(self.ctx.h, self.h, _ptr(grad), lr, beta1, beta2, eps))

    def train(self, cache: Cache, steps: int, batch: int, lr=1e-2, beta1=0.9, beta2=0.99, eps=1e-8, decay=0.92,
              decay_start_frac=0.7, decay_every=25, seed=1, knn_k: int = 0,
              knn_schedule: Sequence[Tuple[float, float]] = ()) -> np.ndarray:
        """Train on the cache's targets: the cell estimate, or with knn_k > 0
        the K-nearest estimate under the staggered schedule knn_schedule =
        [(start fraction of the steps, radius cap in box units), ...]."""
        d = PfTrainDesc(steps, batch, lr, beta1, beta2, eps, decay, decay_start_frac, decay_every, seed)
        if knn_k > 0:
            if not 1 <= len(knn_schedule) <= 8:
                raise ValueError("knn_schedule needs 1..8 (start, radius) stages")
            d.target, d.knn_k, d.knn_stages = 1, knn_k, len(knn_schedule)
            for i, (b, r) in enumerate(knn_schedule):
                d.knn_stage_begin[i], d.knn_radius[i] = b, r
        loss = np.zeros(max(steps, 1), np.float32)
        self.ctx.check(self.ctx.lib.pf_train_field(self.ctx.h, cache.h, C.byref(d), self.h,
                                                   loss.ctypes.data_as(C.c_void_p)))
        return loss[:steps]

    def free(self):
        if self.h:
            self.ctx.lib.pf_field_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def render_neural(ctx: Context, vol: Volume, lights, g: float, cam, spp: int, step_vox: float, seed: int,
                  field: Optional[Field] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    la, n = _lights(lights)
    c = _camera(cam)
    if out is None:
        out = torch.empty(cam.height, cam.width, 3, dtype=torch.float32, device=torch.device("cuda", ctx.device))
    ctx.check(ctx.lib.pf_render_neural(ctx.h, C.byref(vol.s), la, n, float(g), C.byref(c), int(spp), float(step_vox),
                                       int(seed), field.h if field is not None else None, _ptr(out)))
    return out


def render_raymarched(ctx: Context, vol: Volume, lights, g: float, cam, spp: int, step_vox: float, seed: int,
                      field: Optional[Field] = None, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    """Ray marching with the field at every step (pf_render_raymarched)."""
    la, n = _lights(lights)
    c = _camera(cam)
    if out is None:
        out = torch.empty(cam.height, cam.width, 3, dtype=torch.float32, device=torch.device("cuda", ctx.device))
    ctx.check(ctx.lib.pf_render_raymarched(ctx.h, C.byref(vol.s), la, n, float(g), C.byref(c), int(spp),
                                           float(step_vox), int(seed), field.h if field is not None else None,
                                           _ptr(out)))
    return out


def render_pathtraced(ctx: Context, vol: Volume, lights, g: float, cam, spp: int, max_bounces: int = 16, seed: int = 1,
                      use_rr: bool = True, out: Optional[torch.Tensor] = None) -> torch.Tensor:
    la, n = _lights(lights)
    c = _camera(cam)
    if out is None:
        out = torch.empty(cam.height, cam.width, 3, dtype=torch.float32, device=torch.device("cuda", ctx.device))
    ctx.check(ctx.lib.pf_render_pathtraced(ctx.h, C.byref(vol.s), la, n, float(g), C.byref(c), int(spp),
                                           int(max_bounces), int(seed), int(use_rr), _ptr(out)))
    return out


def image_rmse(ctx: Context, a: torch.Tensor, b: torch.Tensor) -> float:
    _need(a, torch.float32, name="a")
    _need(b, torch.float32, a.numel(), "b")
    out = C.c_double()
    ctx.check(ctx.lib.pf_image_rmse(ctx.h, _ptr(a), _ptr(b), a.numel(), C.byref(out)))
    return out.value


def field_encode(ctx: Context, q: torch.Tensor, in_freqs: int = 12) -> torch.Tensor:
    """Frequency encoding of queries q [B, 6] (float32, device): [B, 12 in_freqs]
    features, [input][k][sin, cos] (pf_field_encode)."""
    _need(q, torch.float32, name="q")
    B = q.numel() // 6
    out = torch.empty((B, 12 * in_freqs), dtype=torch.float32, device=q.device)
    ctx.check(ctx.lib.pf_field_encode(ctx.h, _ptr(q), B, int(in_freqs), _ptr(out)))
    return out


class FieldFunction(torch.autograd.Function):
    """Differentiable field evaluation: y = P_phi(q) with gradients w.r.t. the
    flat weight vector w, computed by the library's backward kernel."""

    @staticmethod
    def forward(ctx_, field: Field, q: torch.Tensor, w: torch.Tensor):
        field.set_weights(w.detach().contiguous())
        ctx_.field = field
        ctx_.save_for_backward(q)
        return field.forward(q.contiguous())

    @staticmethod
    def backward(ctx_, gy):
        (q,) = ctx_.saved_tensors
        dw = ctx_.field.backward(q.contiguous(), gy.contiguous().float())
        return None, None, dw
