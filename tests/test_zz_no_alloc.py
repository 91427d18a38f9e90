"""pt_render_noalloc, the render entry point for callers that cannot allocate.

Some callers may not let a library allocate device memory while they render:
a host application that hands out all GPU memory from its own pool at start-up
and forbids later cudaMalloc calls, or a real-time loop that must stay off the
driver's allocator.  pt_render_noalloc keeps its scratch in a fixed array
inside the library instead.  These tests call it through the C ABI and check
that two calls in a row give the image pt_render gives (same kernels, so the
match is to FP32 rounding), that a frame larger than the array is refused, and
that stale contents of the shared array never leak into the next call.

This file is collected last on purpose; it also passes run alone.
"""
import ctypes

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


def _noalloc(pt, scene, nif, cfg, out, err):
    c = pt.make_cfg(cfg)
    return pt.lib().pt_render_noalloc(scene.h, nif.h if nif is not None else None, ctypes.byref(c),
                                      pt._dptr(out), pt._dptr(err), pt._stream(None))


def _check_same(ref, got):
    ref = ref.cpu().numpy()
    got = got.cpu().numpy()
    assert np.all(np.isfinite(got))
    assert np.allclose(got, ref, rtol=1e-5, atol=1e-7)


def test_noalloc_matches_pt_render_two_calls_in_a_row(pt):
    ctx = pt.Context(0)
    scene = pt.Scene(ctx, I.box_scene())
    nif = pt.Nif(ctx, I.nif_init())
    cfg = I.RenderCfg(64, 48, 5, 4)
    ref = pt.render(ctx, scene, nif, cfg)
    ctx.check()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        assert _noalloc(pt, scene, nif, cfg, out, err) == pt.PT_OK
        torch.cuda.synchronize()
        assert int(err.item()) == 0
        _check_same(ref, out)


def test_noalloc_several_chunks_and_no_stale_state(pt):
    """512 x 512 fills the array with one sample, so 3 samples take 3 chunks;
    a smaller frame right after must not see the first call's leftovers."""
    ctx = pt.Context(0)
    scene = pt.Scene(ctx, I.spheres_scene())
    nif = pt.Nif(ctx, I.nif_init(colour="yuv"))
    for cfg in (I.RenderCfg(512, 512, 3, 5), I.RenderCfg(40, 30, 2, 6)):
        ref = pt.render(ctx, scene, nif, cfg)
        ctx.check()
        for _ in range(2):
            out = torch.full_like(ref, float("nan"))
            assert _noalloc(pt, scene, nif, cfg, out, None) == pt.PT_OK
            torch.cuda.synchronize()
            _check_same(ref, out)


def test_noalloc_refuses_frames_beyond_its_array(pt):
    ctx = pt.Context(0)
    scene = pt.Scene(ctx, I.box_scene())
    nif = pt.Nif(ctx, I.nif_init())
    cfg = I.RenderCfg(1024, 1024, 1, 2)      # 1,048,576 pixels > 262,144
    out = torch.zeros((1024, 1024, 3), device="cuda")
    assert _noalloc(pt, scene, nif, cfg, out, None) == pt.PT_EINVAL
    torch.cuda.synchronize()
    assert float(out.abs().max()) == 0.0
    bad = I.RenderCfg(64, 64, 1, 2)
    assert pt.lib().pt_render_noalloc(scene.h, nif.h, ctypes.byref(pt.make_cfg(bad, "bf16")), pt._dptr(out), None,
                                      pt._stream(None)) == pt.PT_EUNSUPPORTED
