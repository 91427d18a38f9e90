"""Render launch sequences are captured into CUDA graphs and replayed when a
render repeats with the same buffers.  A replay must give exactly the image
of direct launches (profiling forces direct launches): with a new sample
offset (a device word, not a captured parameter), after the NIF's colour
matrix changes, for a new scene object, and for cached renders."""
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


def _direct(pt, ctx, fn):
    pt.profile_enable(ctx, True)
    try:
        return fn()
    finally:
        pt.profile_read(ctx)
        pt.profile_enable(ctx, False)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_replay_equals_direct_launches(pt, ctx, prec):
    sc = I.box_scene()
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, I.nif_init(colour="yuv", seed=1))
    cfg = I.RenderCfg(48, 40, 3, 4)
    out = torch.empty((cfg.height, cfg.width, 3), dtype=torch.float32, device="cuda")
    for fs in (0, 0, 5, 9, 5):   # the second call captures, the rest replay with other sample offsets
        a = pt.render(ctx, s, g, cfg, prec, out=out, first_sample=fs).clone()
        b = _direct(pt, ctx, lambda: pt.render(ctx, s, g, cfg, prec, first_sample=fs))
        ctx.check()
        assert torch.equal(a, b), fs
    c = pt.render(ctx, s, g, cfg, prec, out=out, first_sample=0).clone()
    d = pt.render(ctx, s, g, cfg, prec, out=out, first_sample=9).clone()
    assert not torch.equal(c, d)


def test_replay_sees_new_colour_matrix_and_new_scene(pt, ctx):
    cfg = I.RenderCfg(32, 32, 2, 3)
    out = torch.empty((32, 32, 3), dtype=torch.float32, device="cuda")
    nif = I.nif_init(colour="yuv", seed=2)
    g = pt.Nif(ctx, nif)
    s = pt.Scene(ctx, I.box_scene())
    a = pt.render(ctx, s, g, cfg, out=out).clone()
    a2 = pt.render(ctx, s, g, cfg, out=out).clone()
    assert torch.equal(a, a2)
    flat = g.get_params()
    flat[-9:] = np.eye(3, dtype=np.float32).ravel()       # colour matrix -> identity
    g.set_params(flat)
    b = pt.render(ctx, s, g, cfg, out=out).clone()
    b2 = pt.render(ctx, s, g, cfg, out=out).clone()      # captured with the new matrix
    b3 = pt.render(ctx, s, g, cfg, out=out).clone()      # replayed
    want = _direct(pt, ctx, lambda: pt.render(ctx, s, g, cfg))
    assert torch.equal(b, want) and torch.equal(b2, want) and torch.equal(b3, want) and not torch.equal(a, b)
    # a new scene object (the old one freed) must not replay the old scene's graph
    del s
    sc2 = I.box_scene()
    sc2.mat = sc2.mat.copy()
    sc2.mat[:, :3] *= 0.5
    s2 = pt.Scene(ctx, sc2)
    c = pt.render(ctx, s2, g, cfg, out=out).clone()
    c2 = pt.render(ctx, s2, g, cfg, out=out).clone()
    c3 = pt.render(ctx, s2, g, cfg, out=out).clone()
    want2 = _direct(pt, ctx, lambda: pt.render(ctx, s2, g, cfg))
    ctx.check()
    assert torch.equal(c, want2) and torch.equal(c2, want2) and torch.equal(c3, want2) and not torch.equal(b, c)


def test_cached_render_replay(pt, ctx):
    sc = I.box_scene()
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, I.nif_init(colour="yuv", seed=3))
    lo, hi = I.scene_bounds(sc)
    gc = pt.Cache(ctx, I.cache_init(lo, hi, seed=4))
    cfg = I.RenderCfg(32, 24, 2, 5)
    out = torch.empty((32 * 24, 3), dtype=torch.float32, device="cuda")
    for f in range(3):
        gc.train_frame(s, g, 32, 24, f, n_train=2048)
        a = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, precision="bf16", out=out,
                             first_sample=4 * f)[0].clone()
        b = _direct(pt, ctx, lambda: pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2,
                                                      precision="bf16", first_sample=4 * f)[0])
        ctx.check()
        assert torch.equal(a.reshape(b.shape), b), f
