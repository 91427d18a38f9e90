"""Parity at the full sizes of the timed workloads, in the launch
configuration the benchmark times: whole C2, C3 and C5 frames rendered in
one call (one wavefront chunk of 16.8M / 16.8M / 4.2M paths), then a seeded
sample of individual paths (pixel, sample) recomputed by the FP64 oracle and
compared per path under the divergence reading (a path whose hit-ID sequence
differs from the oracle's took another branch at an FP32 vs FP64 decision
and is counted, not compared)."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

from parity_helpers import assert_within_floor, conditioning_table, perturbed_camera, rel_rmse

pytestmark = pytest.mark.gpu

N_SAMPLE = 20000


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def _sample(cfg, seed):
    rng = np.random.default_rng(seed)
    n_pix = cfg.width * cfg.height
    P = rng.integers(0, n_pix, N_SAMPLE)
    S = rng.integers(0, cfg.spp, N_SAMPLE)
    return P, S


def _compare(gL, gids, L, oids, depth_check=None):
    same = np.all(gids == oids, axis=1)
    first = np.where((gids != oids).any(1), (gids != oids).argmax(1), -1)
    res = dict(divergent=float(1 - same.mean()), div_v1=float((first == 0).mean()),
               matched=rel_rmse(gL[same], L[same]), n=int(same.size))
    return res


def _full_frame(pt, ctx, sc, nif, cfg, precision="fp32"):
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, nif) if nif is not None else None
    img, slots, ids = pt.render_pixels(ctx, s, g, cfg, None, precision=precision, want_slots=True, want_ids=True)
    ctx.check()
    assert pt.last_render_schedule(ctx) == "wavefront"
    return img, slots, ids


def _oracle_paths(sc, nif, cfg, P, S, camera=None):
    L, _, oids = O.trace_paths(O.Scene(sc), sc.camera if camera is None else camera, cfg.width, cfg.height,
                               cfg.max_depth, cfg.seed, P, S, nif=O.Nif(nif), want_ids=True)
    return L, oids


def _gpu_paths(pt, ctx, sc, nif, cfg, P, S):
    img, slots, ids = _full_frame(pt, ctx, sc, nif, cfg)
    n_pix = cfg.width * cfg.height
    sl = torch.from_numpy(S * n_pix + P).cuda()
    gL = slots.reshape(-1, 3)[sl].cpu().numpy().astype(np.float64)
    gids = ids.reshape(-1, cfg.max_depth)[sl].cpu().numpy()
    # the frame is the mean of its slots in sample order
    want = slots.double().mean(0).reshape(cfg.height, cfg.width, 3)
    assert torch.allclose(img.double().reshape(cfg.height, cfg.width, 3), want, rtol=1e-5, atol=1e-6)
    return gL, gids


def test_c3_full_frame_sampled_paths(pt, ctx):
    """C3 (heightfield, 1024x1024, 16 spp, depth 6) with the FP32 NIF:
    sampled paths of the whole-frame render against the oracle."""
    sc, nif, cfg = I.make_scene("C3"), I.nif_init(colour="yuv"), I.CONFIGS["C3"]["cfg"]
    P, S = _sample(cfg, 11)
    gL, gids = _gpu_paths(pt, ctx, sc, nif, cfg, P, S)
    L, oids = _oracle_paths(sc, nif, cfg, P, S)
    res = _compare(gL, gids, L, oids)
    print("C3", res)
    assert res["div_v1"] <= 1e-3, res
    assert res["divergent"] <= 2e-3, res
    assert res["matched"] <= 1e-3, res


def test_c2_full_frame_parity_by_specular_vertices(pt, ctx):
    """C2 (256 spheres, 512x512, 64 spp, depth 8, FP32 NIF): sampled paths of
    the whole-frame render against the oracle, binned by the number of
    specular (metal or dielectric) vertices on the oracle's path.

    Reflection off a sphere of radius r seen from distance D multiplies a
    direction error by about 2D/r (Lambertian bounces also inherit the
    normal's error), so an error of one float32 rounding in the path state
    grows bounce by bounce until the path hits another sphere or leaves
    through another part of the sigma = 10 Fourier field.  The floor is
    measured with the oracle itself: the same paths rendered in FP64 from a
    camera moved by one float32 ulp (eye z = 35 -> nextafter) diverge from
    the unperturbed FP64 paths at the rates in the 'floor' columns.  The
    FP32 GPU path is held to that floor per bin (a factor of 3, plus three
    binomial standard deviations of the GPU's divergence count), and to the
    absolute bar (matched-path relative RMSE <= 1e-3) on paths without a
    specular vertex."""
    sc, nif, cfg = I.make_scene("C2"), I.nif_init(colour="yuv"), I.CONFIGS["C2"]["cfg"]
    P, S = _sample(cfg, 11)
    gL, gids = _gpu_paths(pt, ctx, sc, nif, cfg, P, S)
    L, oids = _oracle_paths(sc, nif, cfg, P, S)
    Lp, pids = _oracle_paths(sc, nif, cfg, P, S, camera=perturbed_camera(sc.camera))
    res = _compare(gL, gids, L, oids)
    rows = conditioning_table(sc, oids, L, dict(gpu=(gL, gids), floor=(Lp, pids)))
    print("C2", res)
    for r in rows:
        print("C2 specular vertices", r)
    assert res["div_v1"] <= 1e-3, res
    assert_within_floor(rows)
    assert rows[0]["gpu_matched"] <= 1e-3, rows[0]


def test_c2_full_frame_bf16_paths_follow_fp32(pt, ctx):
    """The C2 frame with the BF16 tensor-core NIF (the benchmark's precision):
    every path takes the same surface hits as with the FP32 NIF (the NIF only
    shades escapes), and the image differs by the NIF's BF16 rounding only."""
    sc, nif, cfg = I.make_scene("C2"), I.nif_init(colour="yuv"), I.CONFIGS["C2"]["cfg"]
    a, _, ida = _full_frame(pt, ctx, sc, nif, cfg, "fp32")
    ida = ida.cpu()
    b, _, idb = _full_frame(pt, ctx, sc, nif, cfg, "bf16")
    assert torch.equal(ida, idb.cpu())
    assert rel_rmse(b.cpu().numpy(), a.cpu().numpy()) <= 1e-2


def test_c5_full_frame_cached_sampled_paths(pt, ctx):
    """The C5 cached render (1024x1024, 4 spp, paths end in a random cache at
    vertex 2, FP32 NIF and cache): sampled paths against the oracle's cached
    paths."""
    sc, nif, cfg = I.make_scene("C5"), I.nif_init(colour="yuv"), I.CONFIGS["C5"]["cfg"]
    lo, hi = I.scene_bounds(sc)
    c = I.cache_init(lo, hi, n_freq=12, hidden=64, n_hidden_layers=5, seed=31)
    rng = np.random.default_rng(32)
    for b in c.b:
        b[:] = rng.normal(0, 0.5, b.shape).astype(np.float32)
    s, g, gc = pt.Scene(ctx, sc), pt.Nif(ctx, nif), pt.Cache(ctx, c)
    _, slots, _, ids = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, want_slots=True,
                                        want_ids=True)
    ctx.check()
    assert pt.last_render_schedule(ctx) == "wavefront"
    P, S = _sample(cfg, 12)
    n_pix = cfg.width * cfg.height
    sl = torch.from_numpy(S * n_pix + P).cuda()
    gL = slots.reshape(-1, 3)[sl].cpu().numpy().astype(np.float64)
    gids = ids.reshape(-1, cfg.max_depth)[sl].cpu().numpy()
    L, _, oids = O.trace_paths(O.Scene(sc), sc.camera, cfg.width, cfg.height, cfg.max_depth, cfg.seed, P, S,
                               nif=O.Nif(nif), cache=O.Cache(c), cache_vertex=2, want_ids=True)
    res = _compare(gL, gids, L, oids)
    print("C5", res)
    assert np.all(gids[:, 2:] == -2)
    assert res["divergent"] <= 2e-3, res
    assert res["matched"] <= 1e-4, res
