"""What the learned part buys: on the data-source scene (thresholded fBm,
albedo 0.95, two point lights), a photon field trained on the GPU photon
caches by the library's own forward/backward kernels lowers the RMSE of the
neural render against a high-spp path-traced reference, compared with the
same renderer without the field (direct light only, L_i = 0) and with the
untrained (Kaiming-initialised) field."""
import numpy as np
import pytest
import torch

from paper_2304_07338_b300 import api, inputs as I

pytestmark = pytest.mark.gpu


def test_trained_field_beats_no_field_and_untrained(pf_ctx):
    sc = I.scene_judge(48, 64, 64, 64)
    vol = api.Volume.from_inputs(sc.volume)
    vol.attach_brick_majorants(pf_ctx)
    g = 0.0
    ref = api.render_pathtraced(pf_ctx, vol, sc.lights, g, sc.camera, 2048, 16, seed=1)
    cache = api.build_photon_cache(pf_ctx, vol, sc.lights, sc.g_set, 1 << 17, 16, 16, seed=2)
    untrained = api.Field(pf_ctx, 12, 64, 4, "bf16", 5.0, seed=3)
    trained = api.Field(pf_ctx, 12, 64, 4, "bf16", 5.0, seed=3)
    loss = trained.train(cache, steps=400, batch=16384, lr=1e-2, seed=4)
    assert loss[-20:].mean() < 0.3 * loss[:5].mean()

    def err(field):
        img = api.render_neural(pf_ctx, vol, sc.lights, g, sc.camera, 64, 0.0, seed=5, field=field)
        return api.image_rmse(pf_ctx, img, ref)

    e_none, e_untrained, e_trained = err(None), err(untrained), err(trained)
    pf_ctx.sync()
    print("rmse: direct only %.4g, untrained %.4g, trained %.4g" % (e_none, e_untrained, e_trained))
    assert e_trained < 0.8 * e_none, (e_trained, e_none)
    assert e_trained < e_untrained
