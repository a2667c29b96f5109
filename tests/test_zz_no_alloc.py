"""The allocation-free path-tracer entry point (pf_render_pathtraced_noalloc).

It exists for callers that cannot allocate device memory while rendering (a
host application owning the whole device budget, a plug-in barred from
allocating in its frame loop, code that must avoid the synchronisation
cudaMalloc / cudaFree can cause).  It keeps its scratch in a fixed file-scope
device array.  Checked through the C ABI: two calls in a row reproduce the
allocating pf_render_pathtraced bit for bit (the path tracer's tolerance),
and an image larger than the static scratch is refused with a message.
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
