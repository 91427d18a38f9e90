"""The two path schedules of a render chunk (Section 3.1) compute the same
paths: the wavefront schedule (one traversal and one shading launch per
vertex, compacted queues between them) and the path-per-thread schedule (one
launch, each thread follows whole paths).  Per-path radiance, hit IDs,
vertex records and ray counts agree bit for bit across scenes with spheres,
quads and triangles, NIF and constant environments, emitters, Russian
roulette, the BF16 NIF and the radiance cache; both agree with the FP64
oracle per path.  The traversal work agrees bit for bit where both
schedules trace every ray on its own (pixel lists); a whole image's camera
rays walk the tree as warp packets in the wavefront schedule, whose work
counts test_gpu_work_counts checks."""
import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

from parity_helpers import rel_rmse

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


def _both(pt, ctx, fn):
    """Run fn(schedule) for both schedules: the outputs with the ray counts per
    vertex, and the traversal work."""
    out, work = {}, {}
    for sched in ("wavefront", "paths"):
        r = fn(sched)
        ctx.check()
        out[sched] = [None if x is None else x.cpu().numpy() for x in r] + \
                     [pt.last_render_counts(ctx, r[-1].shape[-1] if r[-1] is not None else 1)]
        work[sched] = pt.last_render_work(ctx)
    return out["wavefront"], out["paths"], work["wavefront"], work["paths"]


SCENES = {
    "box_nif": (lambda: I.make_scene("C1"), I.RenderCfg(48, 40, 3, 5), "nif"),
    "spheres_nif": (lambda: I.spheres_scene(64), I.RenderCfg(40, 32, 2, 8), "nif"),
    "heightfield_const": (lambda: I.heightfield_scene(32, n_spheres=8, env_const=[0.6, 0.7, 0.9]),
                          I.RenderCfg(40, 32, 2, 6), None),
    "furnace_emitting": (lambda: I.furnace_sphere_inside(0.5), I.RenderCfg(16, 12, 4, 7), None),
    "box_rr": (lambda: I.make_scene("C1"), I.RenderCfg(48, 40, 3, 8, rr=True, rr_start=2), "nif"),
}


@pytest.mark.parametrize("as_list", [False, True])
@pytest.mark.parametrize("name", list(SCENES))
def test_schedules_bit_identical(pt, ctx, name, as_list):
    """The whole image (camera rays in warp packets in the wavefront
    schedule), and every pixel as a list (every ray on its own in both
    schedules: the same work too)."""
    make, cfg, env = SCENES[name]
    sc = make()
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, I.nif_init()) if env == "nif" else None
    pix = torch.arange(cfg.width * cfg.height, dtype=torch.int64, device="cuda") if as_list else None
    a, b, wa, wb = _both(pt, ctx, lambda sched: pt.render_pixels(ctx, s, g, cfg, pix, want_slots=True,
                                                                 want_ids=True, schedule=sched))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert a[-1][0] == cfg.width * cfg.height * cfg.spp   # every path traced its primary ray
    if as_list:
        assert wa == wb


def test_schedules_bit_identical_bf16_nif(pt, ctx):
    """Escapes shaded by the tensor-core NIF: each escape's result does not
    depend on its place in the escape queue."""
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init(colour="yuv"))
    cfg = I.RenderCfg(64, 48, 2, 4)
    a, b, _, _ = _both(pt, ctx, lambda sched: pt.render_pixels(ctx, s, g, cfg, None, precision="bf16",
                                                               want_slots=True, want_ids=True, schedule=sched))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_schedules_bit_identical_cached_with_records(pt, ctx, precision):
    """Records at vertex 1 and cache queries at vertex 2, on a pixel list."""
    sc = I.make_scene("C1")
    lo, hi = I.scene_bounds(sc)
    c = I.cache_init(lo, hi, n_freq=12, hidden=64, n_hidden_layers=5, seed=9)
    s, g, gc = pt.Scene(ctx, sc), pt.Nif(ctx, I.nif_init(colour="yuv")), pt.Cache(ctx, c)
    cfg = I.RenderCfg(64, 64, 3, 5)
    pixels = torch.from_numpy(np.arange(0, 64 * 64, 5, dtype=np.int64)).cuda()
    a, b, wa, wb = _both(pt, ctx, lambda sched: pt.render_cached(ctx, s, g, cfg, pixels, cache=gc, cache_vertex=2,
                                                                 rec_vertex=1, precision=precision, want_slots=True,
                                                                 want_ids=True, schedule=sched))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert wa == wb


def test_paths_schedule_beyond_one_wave_and_chunked(pt, ctx):
    """More paths than the path kernel keeps resident (grid-stride), and
    several chunks with a sample offset."""
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init())
    cfg = I.RenderCfg(512, 384, 1, 3)
    a = pt.render(ctx, s, g, cfg, schedule="wavefront").cpu().numpy()
    b = pt.render(ctx, s, g, cfg, schedule="paths").cpu().numpy()
    cfg2 = I.RenderCfg(96, 64, 6, 4)
    c = pt.render(ctx, s, g, cfg2, chunk_slots=96 * 64 * 2, first_sample=5, schedule="wavefront").cpu().numpy()
    d = pt.render(ctx, s, g, cfg2, chunk_slots=96 * 64 * 2, first_sample=5, schedule="paths").cpu().numpy()
    ctx.check()
    assert np.array_equal(a, b)
    assert np.array_equal(c, d)


@pytest.mark.parametrize("schedule", ["wavefront", "paths"])
def test_each_schedule_matches_oracle_per_path(pt, ctx, schedule):
    """Box scene with the FP32 NIF and roulette: per-path radiance against
    the oracle, paths whose hit sequence differs (an FP32 vs FP64 decision
    flipped) counted and bounded."""
    sc, nif = I.make_scene("C1"), I.nif_init()
    cfg = I.RenderCfg(40, 40, 2, 6, rr=True, rr_start=3)
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    img, slots, ids = pt.render_pixels(ctx, s, g, cfg, None, want_slots=True, want_ids=True, schedule=schedule)
    ctx.check()
    r = O.render(O.Scene(sc), cfg, O.Nif(nif), want_slots=True, want_ids=True)
    gslots = slots.cpu().numpy().transpose(1, 0, 2)
    gids = ids.cpu().numpy().transpose(1, 0, 2)
    same = np.all(gids == r["ids"], axis=2)
    assert same.mean() >= 0.998
    assert rel_rmse(gslots[same], r["slots"][same]) <= 1e-3
    assert rel_rmse(img.cpu().numpy(), r["image"]) <= 2e-3


def test_schedule_argument_checked(pt, ctx):
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init())
    c = pt.make_cfg(I.RenderCfg(8, 8, 1, 2))
    c.schedule = 3
    out = torch.empty((8, 8, 3), dtype=torch.float32, device="cuda")
    st = pt.lib().pt_render(ctx.h, s.h, g.h, None, ctypes.byref(c), pt._dptr(out), None)
    assert st == pt.PT_EINVAL
    ctx.check()


def test_last_render_schedule_reported(pt, ctx):
    """The automatic choice takes the path kernel for a chunk that fits one
    resident wave; a replayed (graph-captured) render reports its own
    schedule, not the one of the render before it."""
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init())
    small = I.RenderCfg(16, 16, 1, 3)
    for _ in range(3):   # first sight, capture, replay
        pt.render(ctx, s, g, small)
        assert pt.last_render_schedule(ctx) == "paths"
        pt.render(ctx, s, g, small, schedule="wavefront")
        assert pt.last_render_schedule(ctx) == "wavefront"
    pt.render(ctx, s, g, I.RenderCfg(512, 384, 1, 2), schedule="paths")
    assert pt.last_render_schedule(ctx) == "paths"
    ctx.check()


def test_kernel_launch_counter(pt, ctx):
    """pt_kernel_launches counts every kernel a render runs, on direct
    launches, on the launch that captures a graph and on graph replays: one
    sample-offset write, per vertex a traversal and a shading kernel (or one
    path kernel), the NIF at the escapes and the reduction."""
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init())
    cfg = I.RenderCfg(16, 16, 1, 3)
    out = torch.empty((16, 16, 3), dtype=torch.float32, device="cuda")
    for sched, want in (("wavefront", 1 + 2 * 3 + 1 + 1), ("paths", 1 + 1 + 1 + 1)):
        for _ in range(3):   # first sight (direct), capture + replay, replay
            k0 = pt.kernel_launches()
            pt.render(ctx, s, g, cfg, out=out, schedule=sched)
            torch.cuda.synchronize()
            assert pt.kernel_launches() - k0 == want, sched
    ctx.check()


@pytest.mark.parametrize("schedule", ["wavefront", "paths"])
def test_tiled_camera_order_same_paths(pt, ctx, schedule):
    """A whole image with W % 8 == 0 and H % 4 == 0 takes its camera rays in
    8x4-pixel tiles; an explicit list of all pixels takes them in row order.
    Every path keeps its slot, so radiance and hit IDs agree bit for bit."""
    s = pt.Scene(ctx, I.make_scene("C1"))
    g = pt.Nif(ctx, I.nif_init())
    cfg = I.RenderCfg(64, 48, 3, 5)
    everything = torch.arange(64 * 48, dtype=torch.int64, device="cuda")
    a = pt.render_pixels(ctx, s, g, cfg, None, want_slots=True, want_ids=True, schedule=schedule)
    b = pt.render_pixels(ctx, s, g, cfg, everything, want_slots=True, want_ids=True, schedule=schedule)
    ctx.check()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.mark.parametrize("case", [("spheres", 64, 1), ("spheres", 512, 2), ("spheres", 2048, 3),
                                  ("heightfield", 48, 4), ("heightfield", 96, 5), ("box", 0, 6)])
def test_camera_packets_give_the_per_ray_hits(pt, ctx, case):
    """Whole images, whose camera rays walk the tree as warp packets on the
    wavefront schedule, against the path-per-thread schedule (every ray on
    its own): per-path radiance, hit IDs and ray counts bit for bit over
    scenes of several sizes and seeds (trees from 64 to 18,000 primitives,
    spheres, triangles and quads)."""
    kind, size, seed = case
    if kind == "spheres":
        sc = I.spheres_scene(size, seed)
        env = "nif"
    elif kind == "heightfield":
        sc = I.heightfield_scene(size, n_spheres=16, seed=seed, env_const=(0.7, 0.8, 1.0))
        env = None
    else:
        sc = I.box_scene(seed)
        env = "nif"
    cfg = I.RenderCfg(64, 48, 4, 6, seed=seed)
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, I.nif_init(seed=seed)) if env == "nif" else None
    a, b, wa, wb = _both(pt, ctx, lambda sched: pt.render_pixels(ctx, s, g, cfg, None, want_slots=True,
                                                                 want_ids=True, schedule=sched))
    for x, y in zip(a, b):
        assert np.array_equal(x, y)
    assert a[-1][0] == cfg.width * cfg.height * cfg.spp
    print({case: {"packets": wa, "per_ray": wb}})
