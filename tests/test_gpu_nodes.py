"""The three BVH node forms (packed 48-byte fp16-extent nodes, decoded
64-byte fp32 nodes, quantised 32-byte 8-bit-grid nodes) hold the same tree
and boxes that contain the exact ones, so they find the same closest hits:
renders of the sphere, box and heightfield scenes are bit-identical across
forms and schedules; unknown forms are refused."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2305_20061_gb300 import inputs as I

pytestmark = pytest.mark.gpu

FORMS = ("packed", "decoded", "quant8")


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


@pytest.mark.parametrize("config,cfg", [("C1", I.RenderCfg(64, 64, 4, 4)), ("C2", I.RenderCfg(128, 96, 4, 8)),
                                        ("C3", I.RenderCfg(160, 128, 4, 6))])
def test_node_forms_render_the_same_paths(pt, ctx, config, cfg):
    sc = I.make_scene(config)
    nif = pt.Nif(ctx, I.nif_init(colour="identity" if config == "C1" else "yuv"))
    out, work = {}, {}
    for form in FORMS:
        s = pt.Scene(ctx, sc, node_format=form)
        assert s.info()["node_format"] == FORMS.index(form) + 1
        for sched in ("wavefront", "paths"):
            out[form, sched] = pt.render_pixels(ctx, s, nif, cfg, None, want_slots=True, want_ids=True,
                                                schedule=sched)
            ctx.check()
            work[form, sched] = pt.last_render_work(ctx)
    ref = out["packed", "wavefront"]
    for k, v in out.items():
        for x, y in zip(ref, v):
            assert torch.equal(x, y), k
    # the decoded form holds the packed form's boxes exactly, so it visits the same nodes
    assert work["decoded", "wavefront"] == work["packed", "wavefront"]
    print(config, {k[0]: v for k, v in work.items() if k[1] == "wavefront"})


def test_node_format_argument(pt, ctx):
    sc = I.make_scene("C1")
    assert pt.Scene(ctx, sc).info()["node_format"] == 2          # automatic: a small tree is decoded
    with pytest.raises(KeyError):
        pt.Scene(ctx, sc, node_format="nope")
    d = pt.SceneDesc()
    d.n_mats = len(sc.mat)
    d.mat_type, d.mats = pt._np_ptr(sc.mat_type), pt._np_ptr(sc.mat)
    d.node_format = 7
    h = ctypes.c_void_p()
    assert pt.lib().pt_create_scene(ctx.h, ctypes.byref(d), ctypes.byref(h)) == pt.PT_EINVAL
