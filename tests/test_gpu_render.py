"""GPU parity of the render path (through the C ABI) against the FP64 oracle:
Philox words, camera rays, closest hits, the FP32 NIF, whole renders,
closed-form scenes, chunking, determinism and argument errors."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
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


def rel_rmse(img, ref):
    img = np.asarray(img, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.sqrt(((img - ref) ** 2).sum() / (ref ** 2).sum()))


def subset_pixels(W, H):
    """Deterministic pixel subset (x + 7 y) mod 16 == 0."""
    y, x = np.divmod(np.arange(W * H), W)
    return np.where((x + 7 * y) % 16 == 0)[0].astype(np.int64)


# ----------------------------------------------------------------------------
def test_philox_words_bit_exact(pt, ctx):
    rng = np.random.default_rng(0)
    ctr = rng.integers(0, 2**32, size=(100003, 4), dtype=np.uint64).astype(np.uint32)
    ctr[:3] = [[0, 0, 0, 0], [0xFFFFFFFF] * 4, [0x243F6A88, 0x85A308D3, 0x13198A2E, 0x03707344]]
    for seed, tag in [(0, 0), (0xA4093822, 0x299F31D0), (7, 1)]:
        got = pt.philox(ctx, seed, tag, torch.from_numpy(ctr.view(np.int32)).cuda()).cpu().numpy().view(np.uint32)
        want = O.philox_batch(seed, tag, ctr)
        assert np.array_equal(got, want)
    ctx.check()


@pytest.mark.parametrize("config", ["C1", "C2", "C3"])
def test_primary_rays_match_oracle(pt, ctx, config):
    sc = I.make_scene(config)
    cfg = I.CONFIGS[config]["cfg"]
    s = pt.Scene(ctx, sc)
    n = 50000
    first = cfg.width * cfg.height * (cfg.spp - 1) - 1234  # spans a sample boundary
    org, dirs = pt.primary_rays(ctx, s, cfg, first, n)
    oo, od = O.primary_rays(sc.camera, cfg.width, cfg.height, cfg.seed, np.arange(first, first + n))
    assert np.allclose(org.cpu().numpy(), oo, atol=1e-6)
    assert np.abs(dirs.cpu().numpy() - od).max() < 2e-6
    ctx.check()


@pytest.mark.parametrize("config", ["C1", "C2", "C3"])
def test_primary_hits_match_oracle(pt, ctx, config):
    """Primary-hit primitive IDs agree on >= 99.99% of rays; every mismatch
    is a near-tie (both primitives within 1e-5 relative distance in FP64)."""
    sc = I.make_scene(config)
    cfg = I.CONFIGS[config]["cfg"]
    s = pt.Scene(ctx, sc)
    osc = O.Scene(sc)
    n = 200000
    org, dirs = pt.primary_rays(ctx, s, cfg, 0, n)
    t, prim = pt.trace_rays(ctx, s, org, dirs)
    ctx.check()
    prim = prim.cpu().numpy()
    oo, od = O.primary_rays(sc.camera, cfg.width, cfg.height, cfg.seed, np.arange(n))
    ot, oid = osc.closest_hit(oo, od)
    mism = np.where(prim != oid)[0]
    assert len(mism) <= 1e-4 * n, (config, len(mism))
    hit = oid >= 0
    tg = t.cpu().numpy()
    assert np.allclose(tg[hit & (prim == oid)], ot[hit & (prim == oid)], rtol=2e-5)
    assert (hit == (prim >= 0)).mean() > 0.9999


def test_trace_rays_random_rays(pt, ctx):
    sc = I.random_triangles_scene(3000, seed=1, n_spheres=50, n_quads=30)
    s = pt.Scene(ctx, sc)
    osc = O.Scene(sc)
    rng = np.random.default_rng(2)
    n = 100000
    o = rng.uniform(-2.5, 2.5, (n, 3)).astype(np.float32)
    d = (rng.uniform(-1, 1, (n, 3)) - o).astype(np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    t, prim = pt.trace_rays(ctx, s, torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda())
    ctx.check()
    ot, oid = osc.closest_hit(o.astype(np.float64), d.astype(np.float64))
    prim = prim.cpu().numpy()
    assert (prim == oid).mean() >= 0.9999
    both = (prim == oid) & (oid >= 0)
    assert np.allclose(t.cpu().numpy()[both], ot[both], rtol=1e-4)


def test_bvh_boxes_contain_their_primitives(pt, ctx):
    """Every packed child box, decoded as fp32 origin + fp16 extent, contains
    all primitives beneath it (Section 3.1.4 rounding never shrinks a box)."""
    sc = I.random_triangles_scene(2000, seed=3, n_spheres=40, n_quads=10)
    s = pt.Scene(ctx, sc)
    nodes, root = s.download_bvh()
    nS, nQ = len(sc.sphere), len(sc.quad)
    lo = np.zeros((sc.n_prims, 3))
    hi = np.zeros((sc.n_prims, 3))
    lo[:nS] = sc.sphere[:, :3] - sc.sphere[:, 3:]
    hi[:nS] = sc.sphere[:, :3] + sc.sphere[:, 3:]
    for i in range(nQ):
        a = sc.quad_axis[i]
        u, v = (a + 1) % 3, (a + 2) % 3
        lo[nS + i, a] = hi[nS + i, a] = sc.quad[i, 0]
        lo[nS + i, u], hi[nS + i, u] = sc.quad[i, 1], sc.quad[i, 2]
        lo[nS + i, v], hi[nS + i, v] = sc.quad[i, 3], sc.quad[i, 4]
    tv = sc.vert[sc.tri].astype(np.float64)
    lo[nS + nQ:] = tv.min(1)
    hi[nS + nQ:] = tv.max(1)
    f = nodes.view(np.float32)
    seen = np.zeros(sc.n_prims, bool)

    def half(bits):
        return np.array([bits], np.uint16).view(np.float16).astype(np.float32)[0]

    def visit(ref):
        if ref & 0x80000000:
            p = ref & 0x7FFFFFFF
            seen[p] = True
            return lo[p], hi[p]
        w = nodes[ref]
        boxes = []
        for side in range(2):
            blo = f[ref, 0:3] if side == 0 else f[ref, 3:6]
            e = ([w[6] & 0xFFFF, w[6] >> 16, w[7] & 0xFFFF] if side == 0 else [w[7] >> 16, w[8] & 0xFFFF, w[8] >> 16])
            bhi = np.array([np.float32(blo[a]) + half(e[a]) for a in range(3)], np.float32)
            clo, chi = visit(int(w[9 + side]))
            assert np.all(blo.astype(np.float64) <= clo) and np.all(bhi.astype(np.float64) >= chi)
            boxes.append((clo, chi))
        return np.minimum(boxes[0][0], boxes[1][0]), np.maximum(boxes[0][1], boxes[1][1])

    import sys
    sys.setrecursionlimit(10000)
    visit(root)
    assert seen.all()


# ----------------------------------------------------------------------------
def test_nif_fp32_matches_oracle(pt, ctx):
    """FP32 NIF within 1e-5 relative per channel of the FP64 oracle fed the
    same float32 (u, v); several 128-row tiles plus a ragged tail."""
    nif = I.nif_init()
    g = pt.Nif(ctx, nif)
    uv = I.uniform_uv(128 * 37 + 41, seed=5)
    uv[:4] = [[0, 0], [0.999999, 0.999999], [0.5, 0.5], [0.25, 1e-7]]
    rgb = g.eval(torch.from_numpy(uv).cuda()).cpu().numpy().astype(np.float64)
    ctx.check()
    ref, _ = O.Nif(nif).forward(uv.astype(np.float64))
    rel = np.abs(rgb - ref) / np.abs(ref)
    assert rel.max() <= 1e-5, rel.max()


def test_nif_fp32_yuv_matrix_and_small_shapes(pt, ctx):
    nif = I.nif_init(n_freq=20, hidden=48, n_hidden_layers=2, colour="yuv", seed=3)
    for b in nif.b:
        b[:] = np.random.default_rng(1).normal(0, 0.1, b.shape)
    g = pt.Nif(ctx, nif)
    uv = I.uniform_uv(1000, seed=6)
    rgb = g.eval(torch.from_numpy(uv).cuda()).cpu().numpy()
    ref, _ = O.Nif(nif).forward(uv.astype(np.float64))
    assert (np.abs(rgb - ref) / np.abs(ref)).max() <= 1e-5


def test_nif_empty_batch(pt, ctx):
    g = pt.Nif(ctx, I.nif_init())
    out = g.eval(torch.zeros((0, 2), device="cuda"))
    assert out.shape == (0, 3)


# ----------------------------------------------------------------------------
def _compare_render(pt, ctx, sc, cfg, nif=None, pixels=None, max_div=1e-3, tol=1e-3, max_div_v1=1e-4,
                    max_div_v2=1e-3):
    """Per-path parity with the oracle (same Philox streams).  A path is
    divergent when its hit-ID sequence differs from the oracle's (an FP32 vs
    FP64 decision flipped somewhere).  Asserted: divergence at the primary
    hit <= max_div_v1, by vertex 2 <= max_div_v2, overall <= max_div, and
    the relative RMSE over matched paths <= tol."""
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, nif) if nif is not None else None
    pix_t = None if pixels is None else torch.from_numpy(pixels).cuda()
    img, slots, ids = pt.render_pixels(ctx, s, g, cfg, pix_t, want_slots=True, want_ids=True)
    ctx.check()
    r = O.render(O.Scene(sc), cfg, O.Nif(nif) if nif is not None else None, pixels=pixels, want_slots=True,
                 want_ids=True)
    gslots = slots.cpu().numpy().transpose(1, 0, 2)          # [n_pix, spp, 3]
    gids = ids.cpu().numpy().transpose(1, 0, 2)               # [n_pix, spp, D]
    differ = gids != r["ids"]
    same = ~np.any(differ, axis=2)
    first = np.where(differ.any(2), differ.argmax(2), -1)
    res = dict(overall=rel_rmse(img.cpu().numpy(), r["image"]),
               matched=rel_rmse(gslots[same], r["slots"][same]),
               divergent=float(1.0 - same.mean()),
               div_v1=float((first == 0).mean()),
               div_v2=float(((first == 0) | (first == 1)).mean()),
               n_paths=int(same.size))
    assert res["div_v1"] <= max_div_v1, res
    assert res["div_v2"] <= max_div_v2, res
    assert res["divergent"] <= max_div, res
    assert res["matched"] <= tol, res
    return res


def test_render_box_config_matches_oracle(pt, ctx):
    """Config C1 in full: 64x64, 8 spp, depth 4, random-init FP32 NIF."""
    cfg = I.CONFIGS["C1"]["cfg"]
    res = _compare_render(pt, ctx, I.box_scene(), cfg, nif=I.nif_init())
    assert res["overall"] <= 1e-3, res


def test_render_spheres_reduced_matches_oracle(pt, ctx):
    """The C2 scene (metal, dielectric, Lambertian spheres) at 96x96, 4 spp,
    depth 8, binned by the number of specular vertices on the oracle's path
    and held to the FP64 floor: the same paths rendered by the oracle from a
    camera moved by one float32 ulp (chained reflections off small spheres
    amplify one rounding bounce by bounce, and the escape direction feeds a
    sigma = 10 Fourier field).  Paths without a specular vertex are held to
    matched-path relative RMSE <= 1e-3."""
    from parity_helpers import assert_within_floor, conditioning_table, perturbed_camera
    cfg = I.RenderCfg(96, 96, 4, 8)
    sc, nif = I.spheres_scene(), I.nif_init()
    s = pt.Scene(ctx, sc)
    _, slots, ids = pt.render_pixels(ctx, s, pt.Nif(ctx, nif), cfg, None, want_slots=True, want_ids=True)
    ctx.check()
    gL = slots.cpu().numpy().transpose(1, 0, 2).reshape(-1, 3).astype(np.float64)
    gids = ids.cpu().numpy().transpose(1, 0, 2).reshape(-1, cfg.max_depth)
    r = O.render(O.Scene(sc), cfg, O.Nif(nif), want_slots=True, want_ids=True)
    sp = I.Scene(**{**sc.__dict__, "camera": perturbed_camera(sc.camera)})
    rp = O.render(O.Scene(sp), cfg, O.Nif(nif), want_slots=True, want_ids=True)
    L, oids = r["slots"].reshape(-1, 3), r["ids"].reshape(-1, cfg.max_depth)
    rows = conditioning_table(sc, oids, L, dict(gpu=(gL, gids),
                                                floor=(rp["slots"].reshape(-1, 3), rp["ids"].reshape(-1, cfg.max_depth))))
    for row in rows:
        print("C2 96x96 specular vertices", row)
    first = np.where((gids != oids).any(1), (gids != oids).argmax(1), -1)
    assert (first == 0).mean() <= 1e-4
    assert_within_floor(rows)
    assert rows[0]["gpu_matched"] <= 1e-3, rows[0]


@pytest.mark.parametrize("depth", [2, 3])
def test_render_spheres_shallow_matches_oracle(pt, ctx, depth):
    """One or two bounces off Lambertian, GGX-metal and dielectric spheres:
    per-path radiance matches the oracle to 1e-3 (pins every lobe's weight
    and direction on the GPU)."""
    cfg = I.RenderCfg(128, 128, 4, depth)
    # a single divergent path can carry more image error than all matched
    # paths together, so the matched-path RMSE is the quantity held to 1e-3
    # and divergence is bounded separately
    res = _compare_render(pt, ctx, I.spheres_scene(), cfg, nif=I.nif_init(), max_div=1e-4)
    print(res)


@pytest.mark.parametrize("kind", [I.METAL, I.DIELECTRIC])
def test_furnace_specular_on_gpu(pt, ctx, kind):
    """Specular furnaces on the GPU: dielectric paths gather exactly 0 or 1;
    metal (F0 = 1) paths agree with the oracle path by path."""
    sc = I.furnace_sphere_outside(kind=kind, f0=1.0, roughness=0.3)
    cfg = I.RenderCfg(48, 48, 4, 6)
    res = _compare_render(pt, ctx, sc, cfg, max_div=2e-3, tol=1e-4)
    if kind == I.DIELECTRIC:
        s = pt.Scene(ctx, sc)
        _, slots, _ = pt.render_pixels(ctx, s, None, cfg, None, want_slots=True)
        ctx.check()
        L = slots.cpu().numpy()
        assert np.all((L == 0.0) | (L == 1.0))
    print(res)


def test_render_heightfield_subset_full_size(pt, ctx):
    """The C3 scene at its full render size on the (x + 7y) mod 16 pixel subset."""
    cfg = I.RenderCfg(1024, 1024, 2, 6)
    res = _compare_render(pt, ctx, I.make_scene("C3"), cfg, nif=I.nif_init(), pixels=subset_pixels(1024, 1024))
    print(res)


def test_furnace_closed_form_on_gpu(pt, ctx):
    a, D = 0.5, 6
    sc = I.furnace_sphere_inside(a)
    cfg = I.RenderCfg(32, 32, 4, D)
    s = pt.Scene(ctx, sc)
    img, slots, _ = pt.render_pixels(ctx, s, None, cfg, None, want_slots=True)
    ctx.check()
    want = float(sc.mat[0, 5]) * sum(float(sc.mat[0, 0]) ** k for k in range(D))
    assert np.allclose(slots.cpu().numpy(), want, rtol=1e-5)


def test_furnace_outside_exact_values(pt, ctx):
    sc = I.furnace_sphere_outside(0.25)
    cfg = I.RenderCfg(48, 48, 2, 3)
    s = pt.Scene(ctx, sc)
    _, slots, ids = pt.render_pixels(ctx, s, None, cfg, None, want_slots=True, want_ids=True)
    ctx.check()
    hit = ids.cpu().numpy()[..., 0] >= 0
    L = slots.cpu().numpy()
    assert np.all(L[hit] == np.float32(0.25)) and np.all(L[~hit] == 1.0)


def test_chunking_and_determinism(pt, ctx):
    cfg = I.RenderCfg(40, 30, 6, 5)
    sc = I.box_scene()
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, I.nif_init())
    a = pt.render(ctx, s, g, cfg).cpu().numpy()
    b = pt.render(ctx, s, g, cfg).cpu().numpy()
    c = pt.render(ctx, s, g, cfg, chunk_slots=40 * 30 * 2).cpu().numpy()
    d = pt.render(ctx, s, g, cfg, chunk_slots=1).cpu().numpy()   # rounded up to one sample
    ctx.check()
    assert np.array_equal(a, b) and np.array_equal(a, c) and np.array_equal(a, d)


def test_degenerate_scenes(pt, ctx):
    # no primitives at all: every path escapes at once
    sc = I.furnace_sphere_outside()
    sc.sphere = np.zeros((0, 4), np.float32)
    sc.sphere_mat = np.zeros((0,), np.int32)
    sc.env_const = np.array([0.5, 2.0, 3.0], np.float32)
    s = pt.Scene(ctx, sc)
    img = pt.render(ctx, s, None, I.RenderCfg(7, 5, 3, 4)).cpu().numpy()
    ctx.check()
    assert np.allclose(img, [0.5, 2.0, 3.0], rtol=1e-6)
    # 1x1 image, depth 1, one sample
    s = pt.Scene(ctx, I.box_scene())
    g = pt.Nif(ctx, I.nif_init())
    img = pt.render(ctx, s, g, I.RenderCfg(1, 1, 1, 1)).cpu().numpy()
    ctx.check()
    r = O.render(O.Scene(I.box_scene()), I.RenderCfg(1, 1, 1, 1), O.Nif(I.nif_init()))
    assert np.allclose(img.reshape(-1, 3), r["image"], rtol=1e-5, atol=1e-7)


def test_invalid_arguments(pt, ctx):
    s = pt.Scene(ctx, I.box_scene())
    with pytest.raises(pt.PTError) as e:
        pt.render(ctx, s, None, I.RenderCfg(8, 8, 1, 2))   # NIF environment but no NIF
    assert e.value.status == pt.PT_EINVAL
    with pytest.raises(pt.PTError) as e:
        pt.render(ctx, s, pt.Nif(ctx, I.nif_init()), I.RenderCfg(8, 8, 1, 0))
    assert e.value.status == pt.PT_EINVAL
    bad = I.box_scene()
    bad.quad_mat = bad.quad_mat.copy()
    bad.quad_mat[0] = 99
    with pytest.raises((pt.PTError, AssertionError)):
        pt.Scene(ctx, bad)
    ctx.check()


def test_russian_roulette_per_path_and_unbiased(pt, ctx):
    """Russian roulette on the GPU (Section 3.1: from depth 3, survival
    probability max(tp)).  Inside a closed Lambertian sphere of albedo 1/2
    emitting 1/2 every throughput is a power of two, so the GPU and the
    oracle draw the same survival decisions from the same Philox words and
    every path's radiance agrees exactly; the mean stays 1 - a^D within 4
    sigma (roulette adds variance, not bias)."""
    a, D = 0.5, 10
    sc = I.furnace_sphere_inside(a)
    cfg = I.RenderCfg(32, 24, 8, D, rr=True, rr_start=3)
    _, slots, _ = pt.render_pixels(ctx, pt.Scene(ctx, sc), None, cfg, None, want_slots=True)
    ctx.check()
    got = slots.cpu().numpy().transpose(1, 0, 2).astype(np.float64)
    r = O.render(O.Scene(sc), cfg, want_slots=True)
    assert np.array_equal(got, r["slots"])
    L = got[..., 0].ravel()
    want = 1.0 - a ** D
    assert L.std() > 0 and abs(L.mean() - want) < 4 * L.std() / np.sqrt(L.size)


def test_russian_roulette_box_parity(pt, ctx):
    """Roulette on a general scene: per-path parity with the oracle (same
    Philox words; a decision flips only when FP32 and FP64 throughputs
    straddle the uniform draw)."""
    cfg = I.RenderCfg(32, 32, 2, 8, rr=True, rr_start=3)
    res = _compare_render(pt, ctx, I.box_scene(), cfg, nif=I.nif_init(), max_div=2e-3)
    assert res["matched"] <= 1e-3, res
