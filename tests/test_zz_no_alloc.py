"""pt_render_noalloc, the render entry point for callers that cannot allocate.

Some callers may not let a library allocate device memory while they render:
a host application that hands out all GPU memory from its own pool at start-up
and forbids later cudaMalloc calls, or a real-time loop that must stay off the
driver's allocator.  pt_render_noalloc keeps its scratch in a fixed array
inside the library instead.  These tests call it through the C ABI and check
that two calls in a row give the image pt_render gives (same kernels, so the
match is to FP32 rounding), also for a constant-environment scene without a
network, that a frame larger than the array is refused, that stale contents
of the shared array never leak into the next call, and that calls leave the
device's free memory unchanged, including the first call in a fresh process
under lazy module loading.

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


def test_noalloc_constant_environment_scene(pt):
    """A constant-environment scene (heightfield with spheres, no network):
    the same image as pt_render, with nif = NULL."""
    ctx = pt.Context(0)
    sc = I.heightfield_scene(48, 30, env_const=(1.0, 1.0, 1.0))
    scene = pt.Scene(ctx, sc)
    cfg = I.RenderCfg(96, 64, 3, 6)
    ref = pt.render(ctx, scene, None, cfg)
    ctx.check()
    for _ in range(2):
        out = torch.full_like(ref, float("nan"))
        assert _noalloc(pt, scene, None, cfg, out, None) == pt.PT_OK
        torch.cuda.synchronize()
        _check_same(ref, out)


def test_noalloc_call_leaves_device_memory_unchanged(pt):
    """What the entry point is for: after one call, further calls (here a
    three-chunk frame) change neither the driver's free-memory count nor
    torch's allocator."""
    ctx = pt.Context(0)
    scene = pt.Scene(ctx, I.spheres_scene())
    nif = pt.Nif(ctx, I.nif_init(colour="yuv"))
    cfg = I.RenderCfg(512, 512, 3, 5)
    out = torch.empty((512, 512, 3), device="cuda")
    assert _noalloc(pt, scene, nif, cfg, out, None) == pt.PT_OK
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    for _ in range(2):
        assert _noalloc(pt, scene, nif, cfg, out, None) == pt.PT_OK
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated(), torch.cuda.memory_reserved())
    assert after == before


_FRESH = r"""
import ctypes, json, sys
import torch
sys.path.insert(0, sys.argv[1])
from paper_2305_20061_gb300 import inputs as I
from paper_2305_20061_gb300 import pt
ctx = pt.Context(0)
scene = pt.Scene(ctx, I.box_scene())
nif = pt.Nif(ctx, I.nif_init())
cfg = I.RenderCfg(64, 48, 5, 4)
ref = pt.render(ctx, scene, nif, cfg)
ctx.check()
out = torch.empty_like(ref)
c = pt.make_cfg(cfg)
torch.cuda.synchronize()
free = [torch.cuda.mem_get_info()[0]]
rcs = []
for _ in range(2):
    rcs.append(pt.lib().pt_render_noalloc(scene.h, nif.h, ctypes.byref(c), pt._dptr(out), None, pt._stream(None)))
    torch.cuda.synchronize()
    free.append(torch.cuda.mem_get_info()[0])
print(json.dumps(dict(rcs=rcs, free=free, same=bool(torch.allclose(out, ref, rtol=1e-5, atol=1e-7)))))
"""


def test_first_call_in_a_fresh_process_allocates_nothing(pt):
    """In a new process under lazy module loading, the very first call (and
    the second) leaves the driver's free-memory count unchanged: pt_create
    has already made the driver reserve the array."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, CUDA_MODULE_LOADING="LAZY")
    r = subprocess.run([sys.executable, "-c", _FRESH, root], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    res = json.loads(r.stdout.strip().splitlines()[-1])
    assert res["rcs"] == [pt.PT_OK, pt.PT_OK] and res["same"], res
    assert res["free"][0] == res["free"][1] == res["free"][2], res
