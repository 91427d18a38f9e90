"""Objects built from host arrays while a render is in flight (the context's
own upload stream, which does not wait for other streams): the images of
renders that use them, and of the render they overlapped, equal those of a
plain sequence; building them does not wait for the running render."""
import time

import numpy as np
import pytest
import torch

from paper_2305_20061_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def test_objects_built_during_a_render_give_the_same_images(pt, ctx):
    cfg_a, cfg_b = I.RenderCfg(256, 256, 512, 8), I.RenderCfg(256, 256, 16, 8)   # a: about 13 ms of GPU work
    sa, sb = I.spheres_scene(256, seed=0), I.spheres_scene(256, seed=3)
    na, nb = I.nif_init(colour="yuv", seed=0), I.nif_init(colour="yuv", seed=4)
    # the plain sequence
    ref_a = pt.render(ctx, pt.Scene(ctx, sa), pt.Nif(ctx, na), cfg_a, "bf16").clone()
    ref_b = pt.render(ctx, pt.Scene(ctx, sb), pt.Nif(ctx, nb), cfg_b, "bf16").clone()
    torch.cuda.synchronize()
    ctx.check()
    # b's scene and weights built and uploaded while a renders
    s_a, n_a = pt.Scene(ctx, sa), pt.Nif(ctx, na)
    img_a = pt.render(ctx, s_a, n_a, cfg_a, "bf16")
    t0 = time.perf_counter()
    s_b, n_b = pt.Scene(ctx, sb), pt.Nif(ctx, nb)
    t_build = time.perf_counter() - t0
    img_b = pt.render(ctx, s_b, n_b, cfg_b, "bf16")
    torch.cuda.synchronize()
    t_all = time.perf_counter() - t0
    ctx.check()
    assert torch.equal(img_a, ref_a) and torch.equal(img_b, ref_b)
    print({"build_ms": 1e3 * t_build, "build_and_render_ms": 1e3 * t_all})
    # building b took a small part of the time a's render still had to run (it did not wait for it)
    assert t_build < 0.25 * t_all


def test_scene_destroyed_after_its_render_completes(pt, ctx):
    """pt_destroy_scene and pt_destroy_nif wait for the device: destroying
    the objects of a render still in flight leaves its image intact."""
    cfg = I.RenderCfg(128, 128, 32, 8)
    sc, nif = I.spheres_scene(64, seed=1), I.nif_init(colour="yuv", seed=2)
    ref = pt.render(ctx, pt.Scene(ctx, sc), pt.Nif(ctx, nif), cfg, "bf16").clone()
    torch.cuda.synchronize()
    s, n = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    img = pt.render(ctx, s, n, cfg, "bf16")
    del s, n
    torch.cuda.synchronize()
    ctx.check()
    assert torch.equal(img, ref)
