"""The allocation-free path-tracer entry point (pf_render_pathtraced_noalloc).

It exists for callers that cannot allocate device memory while rendering (a
host application owning the whole device budget, a plug-in barred from
allocating in its frame loop, code that must avoid the synchronisation
cudaMalloc / cudaFree can cause).  It keeps its scratch in a fixed file-scope
device array.  Checked through the C ABI: two calls in a row reproduce the
allocating pf_render_pathtraced bit for bit (the path tracer's tolerance),
also when the image needs several chunks of the static scratch, and inputs
the allocating entry point refuses (a zero light direction, an invalid
brick, an image larger than the static scratch) are refused with a message.
This file sorts last so that a failure here comes after every other test.
"""
import ctypes as C

import numpy as np
import pytest
import torch

from paper_2304_07338_b300 import _lib, api, inputs as I

pytestmark = pytest.mark.gpu


def _call(L, vol, lights, g, cam, spp, max_bounces, seed, out, msg):
    la, n = api._lights(lights)
    c = api._camera(cam)
    stream = torch.cuda.current_stream().cuda_stream
    return L.pf_render_pathtraced_noalloc(C.byref(vol.s), la, n, float(g), C.byref(c), spp, max_bounces, seed, 1,
                                          C.c_void_p(stream), C.c_void_p(out.data_ptr()), msg, len(msg))


def test_noalloc_matches_allocating_path_tracer(pf_ctx):
    L = _lib.load()
    sc = I.scene_judge(32, 48, 36, 8)
    vol = api.Volume.from_inputs(sc.volume)
    vol.attach_brick_majorants(pf_ctx)
    ref = api.render_pathtraced(pf_ctx, vol, sc.lights, 0.5, sc.camera, sc.spp, 16, seed=13)
    pf_ctx.sync()
    msg = C.create_string_buffer(256)
    for _ in range(2):                      # the shared scratch keeps the previous call's contents
        out = torch.full_like(ref, -1.0)
        st = _call(L, vol, sc.lights, 0.5, sc.camera, sc.spp, 16, 13, out, msg)
        assert st == _lib.PF_OK, msg.value
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    assert float(ref.max()) > 0


def test_noalloc_rejects_oversize_and_missing_majorants(pf_ctx):
    L = _lib.load()
    sc = I.scene_judge(16, 8, 8, 1)
    vol = api.Volume.from_inputs(sc.volume)
    msg = C.create_string_buffer(256)
    out = torch.zeros(8, 8, 3, device="cuda")
    st = _call(L, vol, sc.lights, 0.0, sc.camera, 1, 4, 1, out, msg)
    assert st == _lib.PF_ERR_INVALID_ARG and b"majorant" in msg.value
    vol.attach_brick_majorants(pf_ctx)
    big = I.Camera(sc.camera.eye, sc.camera.at, sc.camera.up, 55.0, 2048, 2048)
    st = _call(L, vol, sc.lights, 0.0, big, 1, 4, 1, out, msg)
    assert st == _lib.PF_ERR_INVALID_ARG and b"static scratch" in msg.value


def test_noalloc_several_chunks_match(pf_ctx):
    """1920x1080 at 3 spp: the static array holds the per-pixel accumulator and
    one sample per pixel, so the render runs in three chunks (the allocating
    path in one); the in-order per-pixel sums make the bits equal."""
    L = _lib.load()
    sc = I.scene_judge(16, 1920, 1080, 3)
    vol = api.Volume.from_inputs(sc.volume)
    vol.attach_brick_majorants(pf_ctx)
    ref = api.render_pathtraced(pf_ctx, vol, sc.lights, 0.0, sc.camera, 3, 2, seed=21)
    pf_ctx.sync()
    msg = C.create_string_buffer(256)
    out = torch.full_like(ref, -1.0)
    st = _call(L, vol, sc.lights, 0.0, sc.camera, 3, 2, 21, out, msg)
    assert st == _lib.PF_OK, msg.value
    torch.cuda.synchronize()
    assert float(ref.max()) > 0
    assert torch.equal(out, ref)


def test_noalloc_rejects_what_the_allocating_path_rejects(pf_ctx):
    L = _lib.load()
    sc = I.scene_judge(16, 8, 8, 1)
    vol = api.Volume.from_inputs(sc.volume)
    vol.attach_brick_majorants(pf_ctx)
    msg = C.create_string_buffer(256)
    out = torch.zeros(8, 8, 3, device="cuda")
    zero_dir = [I.Light(I.DIRECTIONAL, (0.0, 0.0, 0.0), (1.0, 1.0, 1.0))]
    st = _call(L, vol, zero_dir, 0.0, sc.camera, 1, 4, 1, out, msg)
    assert st == _lib.PF_ERR_INVALID_ARG and b"direction" in msg.value
    with pytest.raises(api.PfError):
        api.render_pathtraced(pf_ctx, vol, zero_dir, 0.0, sc.camera, 1, 4, seed=1)
    inside = [I.Light(I.POINT, (0.5, 0.5, 0.5), (1.0, 1.0, 1.0))]
    st = _call(L, vol, inside, 0.0, sc.camera, 1, 4, 1, out, msg)
    assert st == _lib.PF_ERR_INVALID_ARG and b"outside" in msg.value
    good = vol.s.brick
    try:
        vol.s.brick = 3                      # not a power of two
        st = _call(L, vol, sc.lights, 0.0, sc.camera, 1, 4, 1, out, msg)
        assert st == _lib.PF_ERR_INVALID_ARG and b"brick" in msg.value
        with pytest.raises(api.PfError):
            api.render_pathtraced(pf_ctx, vol, sc.lights, 0.0, sc.camera, 1, 4, seed=1)
    finally:
        vol.s.brick = good
    ss = vol.s.sigma_scale
    try:
        vol.s.sigma_scale = float("inf")
        st = _call(L, vol, sc.lights, 0.0, sc.camera, 1, 4, 1, out, msg)
        assert st == _lib.PF_ERR_INVALID_ARG and b"sigma_scale" in msg.value
    finally:
        vol.s.sigma_scale = ss
    # a degenerate camera frame (eye == at) is refused by both entry points
    flat = I.Camera((0.5, 0.5, 3.0), (0.5, 0.5, 3.0), (0, 1, 0), 30.0, 8, 8)
    st = _call(L, vol, sc.lights, 0.0, flat, 1, 4, 1, out, msg)
    assert st == _lib.PF_ERR_INVALID_ARG and b"camera" in msg.value
    with pytest.raises(api.PfError):
        api.render_pathtraced(pf_ctx, vol, sc.lights, 0.0, flat, 1, 4, seed=1)
