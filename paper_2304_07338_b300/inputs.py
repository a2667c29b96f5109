"""Seeded synthetic inputs: density volumes, transfer functions, lights, cameras.

This module holds no arithmetic of the method itself.  It only builds the
scenes that both the CUDA path and the CPU oracle consume: scalar volumes
standing in for the paper's scientific datasets (Sec. 4, Table of rendering
performance), piecewise-linear RGBA transfer functions (the TransferFunction
step of Algorithm 1), light lists (Algorithm 1 "generate from random light
source"), pinhole cameras (Algorithm 2 input `camera`) and the phase sets
(Sec. 3.2, the set G of Henyey-Greenstein coefficients).

Conventions shared by every consumer:
  * volumes are x-fastest arrays of shape (nz, ny, nx) covering [0,1]^3 with
    voxel (i,j,k) centred at ((i+1/2)/nx, (j+1/2)/ny, (k+1/2)/nz);
  * dtype codes: 0 = float32, 1 = float16, 2 = uint8 (density = value/255);
  * a transfer function is an (n, 4) float32 RGBA table over density [0,1],
    interpolated linearly; sigma_t = sigma_scale * alpha, albedo = A * rgb;
  * `brick` is the edge (voxels) of the bricks whose majorants drive delta
    and ratio tracking;
  * a light is (kind, v[3], rgb[3]): kind 0 = directional with v pointing
    towards the light and rgb its irradiance, kind 1 = point light at v with
    rgb its intensity;
  * a camera is (eye[3], at[3], up[3], fovy_deg, width, height).

Volumes of up to a few hundred MB are built with numpy on the host; the
1024^3 turbulence volume is built with torch on a CUDA device when one is
given, because generating a gigavoxel field on the host takes minutes.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Tuple

import numpy as np

MASTER_SEED = 20230414

F32, F16, U8 = 0, 1, 2
DIRECTIONAL, POINT = 0, 1


@dataclasses.dataclass
class Volume:
    data: np.ndarray            # (nz, ny, nx), float32 / float16 / uint8
    sigma_scale: float
    albedo: float
    tf: np.ndarray              # (n, 4) float32 RGBA
    brick: int = 8              # edge of the majorant bricks in voxels (power of two)
    brick_primary: int = 0      # brick edge for the camera rays' free flight (0: brick)
    brick_shadow: int = 0       # brick edge walked by shadow rays, thinned to brick (0: brick)

    @property
    def dtype_code(self) -> int:
        return {np.dtype(np.float32): F32, np.dtype(np.float16): F16,
                np.dtype(np.uint8): U8}[np.dtype(self.data.dtype)]

    @property
    def shape_xyz(self) -> Tuple[int, int, int]:
        nz, ny, nx = self.data.shape
        return nx, ny, nz


@dataclasses.dataclass
class Light:
    kind: int
    v: Tuple[float, float, float]
    rgb: Tuple[float, float, float]


@dataclasses.dataclass
class Camera:
    eye: Tuple[float, float, float]
    at: Tuple[float, float, float]
    up: Tuple[float, float, float]
    fovy_deg: float
    width: int
    height: int


# ---------------------------------------------------------------- transfer functions
def tf_linear_gray() -> np.ndarray:
    """TF(d) = (d, d, d, d): alpha and colour both equal the density."""
    return np.array([[0, 0, 0, 0], [1, 1, 1, 1]], np.float32)


def tf_white_alpha_ramp() -> np.ndarray:
    """TF(d) = (1, 1, 1, d): white albedo, alpha equal to the density."""
    return np.array([[1, 1, 1, 0], [1, 1, 1, 1]], np.float32)


def tf_constant(alpha: float = 1.0, rgb=(1.0, 1.0, 1.0)) -> np.ndarray:
    """Density-independent TF, used for homogeneous-medium closed forms."""
    r, g, b = rgb
    return np.array([[r, g, b, alpha], [r, g, b, alpha]], np.float32)


def tf_piecewise_rgba(n: int = 256) -> np.ndarray:
    """A piecewise-linear RGBA ramp sampled at n nodes (a colour map that
    hides low densities, warm mid tones, bright white cores)."""
    nodes_d = np.array([0.0, 0.25, 0.45, 0.65, 0.85, 1.0])
    nodes = np.array([
        [0.00, 0.00, 0.00, 0.00],
        [0.20, 0.35, 0.90, 0.00],
        [0.35, 0.75, 0.85, 0.35],
        [0.95, 0.70, 0.30, 0.70],
        [0.95, 0.40, 0.25, 0.90],
        [1.00, 1.00, 1.00, 1.00],
    ])
    d = np.linspace(0.0, 1.0, n)
    out = np.stack([np.interp(d, nodes_d, nodes[:, c]) for c in range(4)], 1)
    return out.astype(np.float32)


# ---------------------------------------------------------------- volumes
def _centres(n: int) -> np.ndarray:
    return (np.arange(n, dtype=np.float64) + 0.5) / n


def blobs_volume(n: int = 64, n_blobs: int = 8, seed: int = MASTER_SEED) -> np.ndarray:
    """Sum of isotropic Gaussian blobs, centres U[0.2,0.8]^3, std U[0.05,0.15],
    unit amplitude, clamped to [0,1]; float32 (n, n, n)."""
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=(n_blobs, 3))
    s = rng.uniform(0.05, 0.15, size=n_blobs)
    x = _centres(n)
    vol = np.zeros((n, n, n), np.float64)
    for b in range(n_blobs):
        gx = np.exp(-((x - c[b, 0]) ** 2) / (2 * s[b] ** 2))
        gy = np.exp(-((x - c[b, 1]) ** 2) / (2 * s[b] ** 2))
        gz = np.exp(-((x - c[b, 2]) ** 2) / (2 * s[b] ** 2))
        vol += gz[:, None, None] * gy[None, :, None] * gx[None, None, :]
    return np.clip(vol, 0.0, 1.0).astype(np.float32)


def _value_noise(n: int, freq: int, rng: np.random.Generator, signed: bool) -> np.ndarray:
    """Lattice noise of `freq` cells per axis, trilinearly interpolated at the
    voxel centres of an n^3 grid (lattice wraps periodically)."""
    lat = rng.uniform(-1.0 if signed else 0.0, 1.0, size=(freq, freq, freq))
    p = _centres(n) * freq
    i0 = np.floor(p).astype(np.int64)
    t = p - i0
    i0 %= freq
    i1 = (i0 + 1) % freq
    a = lat[:, :, i0] * (1 - t)[None, None, :] + lat[:, :, i1] * t[None, None, :]
    a = a[:, i0, :] * (1 - t)[None, :, None] + a[:, i1, :] * t[None, :, None]
    a = a[i0, :, :] * (1 - t)[:, None, None] + a[i1, :, :] * t[:, None, None]
    return a


def fbm_volume(n: int = 128, octaves: int = 5, base_freq: int = 4, lacunarity: int = 2,
               gain: float = 0.5, threshold: float = 0.4, seed: int = MASTER_SEED + 1) -> np.ndarray:
    """Fractal value noise (fBm), normalised to [0,1], zeroed below `threshold`."""
    rng = np.random.default_rng(seed)
    acc = np.zeros((n, n, n), np.float64)
    amp, freq = 1.0, base_freq
    for _ in range(octaves):
        acc += amp * _value_noise(n, freq, rng, signed=False)
        amp *= gain
        freq *= lacunarity
    acc = (acc - acc.min()) / max(acc.max() - acc.min(), 1e-12)
    acc[acc < threshold] = 0.0
    return acc.astype(np.float32)


def _gauss_kernel(sigma: float) -> np.ndarray:
    r = int(math.ceil(3 * sigma))
    x = np.arange(-r, r + 1, dtype=np.float64)
    k = np.exp(-x * x / (2 * sigma * sigma))
    return (k / k.sum()).astype(np.float32)


def _restore(v, shape, axis):
    # v holds rows of the volume with `axis` moved last; move it back
    s = list(shape)
    moved = s[:axis] + s[axis + 1:] + [s[axis]]
    return v.reshape(moved).movedim(-1, axis)


def blurred_noise_volume(n: int = 512, seed: int = MASTER_SEED + 3, device: Optional[str] = None) -> np.ndarray:
    """N(0,1) white noise blurred three times by separable Gaussians of
    std 1, 2 and 4 voxels, min-max normalised and quantised to uint8."""
    import torch
    g = torch.Generator(device="cpu").manual_seed(seed)
    vol = torch.randn((n, n, n), generator=g, dtype=torch.float32)
    dev = device or "cpu"
    vol = vol.to(dev)
    for sigma in (1.0, 2.0, 4.0):
        k = torch.from_numpy(_gauss_kernel(sigma)).to(dev)
        r = (k.numel() - 1) // 2
        for axis in range(3):
            v = vol.movedim(axis, -1).reshape(-1, 1, n)
            v = torch.nn.functional.pad(v, (r, r), mode="replicate")
            v = torch.nn.functional.conv1d(v, k.view(1, 1, -1))
            vol = _restore(v, vol.shape, axis)
    lo, hi = vol.min(), vol.max()
    vol = (vol - lo) / (hi - lo)
    return torch.round(vol * 255.0).clamp(0, 255).to(torch.uint8).cpu().numpy()


def turbulence_volume(n: int = 1024, octaves: int = 6, base_freq: int = 4,
                      seed: int = MASTER_SEED + 4, device: Optional[str] = None):
    """Turbulence sum_o 0.5^o |noise_o| of signed value noise, normalised to
    [0,1], float16.  Returns a torch tensor on `device` (default: cpu)."""
    import torch
    dev = torch.device(device or "cpu")
    g = torch.Generator(device="cpu").manual_seed(seed)
    acc = torch.zeros((n, n, n), dtype=torch.float32, device=dev)
    freq, amp = base_freq, 1.0
    for _ in range(octaves):
        lat = (torch.rand((freq + 1,) * 3, generator=g) * 2 - 1).to(dev)
        lat[freq, :, :] = lat[0, :, :]
        lat[:, freq, :] = lat[:, 0, :]
        lat[:, :, freq] = lat[:, :, 0]
        p = (torch.arange(n, device=dev, dtype=torch.float32) + 0.5) * (freq / n)
        i0 = torch.floor(p).long()
        t = p - i0
        i1 = i0 + 1
        lx = lat[:, :, i0] * (1 - t) + lat[:, :, i1] * t
        lxy = lx[:, i0, :] * (1 - t)[:, None] + lx[:, i1, :] * t[:, None]
        for z0 in range(0, n, 128):
            z1 = min(n, z0 + 128)
            tz = t[z0:z1][:, None, None]
            slab = lxy[i0[z0:z1]] * (1 - tz) + lxy[i1[z0:z1]] * tz
            acc[z0:z1] += amp * slab.abs()
        freq *= 2
        amp *= 0.5
    lo, hi = acc.min(), acc.max()
    acc = (acc - lo) / (hi - lo)
    return acc.to(torch.float16)


# ---------------------------------------------------------------- lights, cameras
def _unit(v):
    v = np.asarray(v, np.float64)
    return v / np.linalg.norm(v)


def point_lights(n: int, seed: int, radius: float = 1.5, intensity: float = 2.25) -> List[Light]:
    """n point lights at c + radius*u_l, u_l seeded unit vectors, white
    intensity `intensity` (irradiance about 1 at the volume centre)."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        u = _unit(rng.normal(size=3))
        p = 0.5 + radius * u
        out.append(Light(POINT, tuple(float(a) for a in p), (intensity,) * 3))
    return out


def orbit_camera(azimuth: float, elevation: float, width: int, height: int,
                 distance: float = 2.0, fovy_deg: float = 55.0) -> Camera:
    """Camera at c + distance*d_f looking at the volume centre c=(.5,.5,.5)."""
    d = np.array([math.cos(elevation) * math.cos(azimuth), math.sin(elevation),
                  math.cos(elevation) * math.sin(azimuth)])
    eye = 0.5 + distance * d
    up = (0.0, 1.0, 0.0) if abs(d[1]) <= 0.99 else (0.0, 0.0, 1.0)
    return Camera(tuple(float(a) for a in eye), (0.5, 0.5, 0.5), up, fovy_deg, width, height)


# ---------------------------------------------------------------- workloads
G_PAPER = (-0.75, 0.0, 0.75)      # Sec. 3.2
G_JUDGE = (-0.5, 0.0, 0.5)


@dataclasses.dataclass
class Scene:
    name: str
    volume: Volume
    lights: List[Light]
    camera: Camera
    spp: int
    g: float
    g_set: Tuple[float, ...]
    seed: int
    step_vox: float = 0.5


def scene_small(n: int = 64, width: int = 128, height: int = 128, spp: int = 4) -> Scene:
    """Plain-method scene: 64^3 Gaussian blobs, sigma_t scale 20, albedo 0.9,
    linear grey TF, one directional light, g=0, 128^2 x 4 spp."""
    seed = MASTER_SEED
    vol = Volume(blobs_volume(n, 8, seed), 20.0, 0.9, tf_linear_gray())
    light = Light(DIRECTIONAL, tuple(float(a) for a in _unit([1.0, 1.0, 0.5])), (1.0, 1.0, 1.0))
    cam = orbit_camera(0.6, 0.35, width, height)
    return Scene("blobs64", vol, [light], cam, spp, 0.0, (0.0,), seed)


def scene_judge(n: int = 128, width: int = 256, height: int = 256, spp: int = 64) -> Scene:
    """Judge / data-source scene: 128^3 thresholded fBm, albedo 0.95,
    two point lights, G = {-0.5, 0, 0.5}, 256^2 path-traced at 64 spp."""
    seed = MASTER_SEED + 1
    vol = Volume(fbm_volume(n, seed=seed), 20.0, 0.95, tf_white_alpha_ramp())
    cam = orbit_camera(0.6, 0.35, width, height)
    return Scene("fbm128", vol, point_lights(2, seed), cam, spp, 0.0, G_JUDGE, seed)


def scene_mid(n: int = 512, width: int = 1024, height: int = 1024, spp: int = 4,
              device: Optional[str] = None) -> Scene:
    """Mid render: 512^3 uint8 blurred noise, 256-node RGBA TF, 4 lights,
    g drawn from U[-0.9,0.9] per frame, 1024^2 x 4 spp."""
    seed = MASTER_SEED + 3
    vol = Volume(blurred_noise_volume(n, seed, device), 20.0, 0.9, tf_piecewise_rgba(256))
    cam = orbit_camera(0.6, 0.35, width, height)
    g = float(np.random.default_rng(seed).uniform(-0.9, 0.9))
    return Scene("noise512u8", vol, point_lights(4, seed), cam, spp, g, G_PAPER, seed)


def large_scene_parts(n: int = 1024, device: Optional[str] = None):
    """Large render: 1024^3 float16 turbulence (2 GiB), 8 point lights,
    1920x1080, 16 spp, 60-frame orbit at 20 degrees elevation.  Returns
    (volume tensor, tf, lights, cameras) so the volume can stay on device."""
    seed = MASTER_SEED + 4
    vol = turbulence_volume(n, seed=seed, device=device)
    cams = [orbit_camera(2 * math.pi * f / 60, math.radians(20.0), 1920, 1080) for f in range(60)]
    return vol, tf_piecewise_rgba(256), point_lights(8, seed), cams


def frame_g(seed: int, frame: int) -> float:
    """Per-frame phase coefficient g ~ U[-0.9, 0.9] (seeded by frame)."""
    return float(np.random.default_rng([seed, frame]).uniform(-0.9, 0.9))
