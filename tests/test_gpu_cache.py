"""GPU parity of the neural radiance cache (through the C ABI) against the
FP64 oracle: the fused evaluation kernel, the relative-L2 loss and gradient,
vertex records and training targets, cached renders (per path and in the
closed furnace), and the online training step."""
import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

from parity_helpers import rel_rmse

pytestmark = pytest.mark.gpu

TRAIN_SAMPLE_BASE = 1 << 30   # sample index of the training paths of frame 0


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def _cache(lo, hi, seed=3, J=12, L=5, bias_std=0.1):
    c = I.cache_init(lo, hi, n_freq=J, hidden=64, n_hidden_layers=L, seed=seed)
    rng = np.random.default_rng(seed + 100)
    for b in c.b:
        b[:] = rng.normal(0, bias_std, b.shape).astype(np.float32)
    return c


def _queries(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    x = rng.uniform(lo, hi, (n, 3))
    d = rng.normal(0, 1, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    nn = rng.normal(0, 1, (n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    return np.concatenate([x, d, nn], 1).astype(np.float32)


# ----------------------------------------------------------------------------
@pytest.mark.parametrize("J,L,n", [(12, 5, 1000), (12, 5, 1), (4, 2, 385), (15, 7, 300)])
def test_cache_eval_matches_oracle(pt, ctx, J, L, n):
    """FP32 fused MLP vs FP64 on the same FP32 queries, including positions on
    the box faces; tiles of 128 with a ragged tail."""
    lo, hi = np.array([-3.0, 0.5, -1.0], np.float32), np.array([2.0, 4.0, 6.5], np.float32)
    c = _cache(lo, hi, seed=J + L, J=J, L=L)
    q = _queries(n, lo, hi, seed=n)
    q[: min(n, 6), :3] = np.array([lo, hi, lo, hi, lo, hi])[: min(n, 6)]
    got = pt.Cache(ctx, c).eval(torch.from_numpy(q).cuda()).cpu().numpy()
    ctx.check()
    want = O.Cache(c).forward(q.astype(np.float64))
    scale = np.abs(want).max()
    assert np.abs(got - want).max() <= 1e-5 * scale + 1e-6, np.abs(got - want).max()


def test_cache_eval_empty(pt, ctx):
    c = _cache([0, 0, 0], [1, 1, 1])
    out = pt.Cache(ctx, c).eval(torch.zeros((0, 9), device="cuda"))
    ctx.check()
    assert out.shape == (0, 3)


def _bf16(x):
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _bf16_cache_model(c, q):
    """Rounding model of the tensor-core cache: BF16 encoding, weights and
    activations, biases as BF16 hi + lo, FP64 sums standing in for FP32
    accumulation, FP32 output bias."""
    q = q.astype(np.float64)
    lo, hi = c.lo.astype(np.float64), c.hi.astype(np.float64)
    p = (q[:, :3] - lo) / (hi - lo)
    feats = []
    for a in range(3):
        ang = np.pi * p[:, a:a + 1] * (2.0 ** np.arange(c.n_freq))[None]
        feats += [np.sin(ang), np.cos(ang)]
    x = _bf16(np.concatenate(feats + [q[:, 3:9]], 1).astype(np.float32)).astype(np.float64)
    for W, b in zip(c.W[:-1], c.b[:-1]):
        bh = _bf16(b).astype(np.float64)
        bl = _bf16((b.astype(np.float64) - bh).astype(np.float32)).astype(np.float64)
        x = _bf16(np.maximum(x @ _bf16(W).astype(np.float64).T + bh + bl, 0).astype(np.float32)).astype(np.float64)
    return x @ _bf16(c.W[-1]).astype(np.float64).T + c.b[-1].astype(np.float64)


@pytest.mark.parametrize("n", [1, 129, 128 * 152 * 4 * 2 + 77])
def test_bf16_cache_matches_rounding_model(pt, ctx, n):
    """The tcgen05 cache kernel against a numpy model of its own rounding, and
    its error against the FP64 oracle (reported; a loose bound guards against
    gross errors)."""
    lo, hi = np.array([-1.0, -0.2, -1.0], np.float32), np.array([1.0, 0.2, 1.0], np.float32)
    c = _cache(lo, hi, seed=41)
    q = _queries(n, lo, hi, seed=n + 3)
    gc = pt.Cache(ctx, c)
    got = gc.eval(torch.from_numpy(q).cuda(), precision="bf16").cpu().numpy().astype(np.float64)
    ctx.check()
    ref = _bf16_cache_model(c, q)
    scale = np.abs(ref).max()
    err = np.abs(got - ref)
    assert np.median(err) <= 2e-3 * scale and err.max() <= 3e-2 * scale, (np.median(err) / scale, err.max() / scale)
    exact = O.Cache(c).forward(q.astype(np.float64))
    rel = float(np.sqrt(((got - exact) ** 2).sum() / (exact ** 2).sum()))
    print(f"BF16 cache vs FP64 oracle: relative RMSE {rel:.3e} over {n} queries")
    assert rel <= 5e-2


def test_bf16_cached_render_close_to_fp32(pt, ctx):
    """A cached render with the BF16 NIF and BF16 cache against the same render
    in FP32: same paths, image relative RMSE from the two networks' rounding."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = _cache(lo, hi, seed=43, bias_std=0.5)
    cfg = I.RenderCfg(64, 64, 4, 4, 0)
    s, gc = pt.Scene(ctx, sc), pt.Cache(ctx, c)
    nif_tc = I.nif_init(colour="yuv")
    g = pt.Nif(ctx, nif_tc)
    a = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, precision="bf16")[0].cpu().numpy()
    b = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, precision="fp32")[0].cpu().numpy()
    ctx.check()
    rel = rel_rmse(a, b)
    print(f"BF16 vs FP32 cached render: relative RMSE {rel:.3e}")
    assert rel <= 2e-2


def test_cache_loss_grad_matches_oracle(pt, ctx):
    """Relative L2 with the prediction held constant in the denominator;
    20% of the rows masked; 3000 rows (ragged against the 128-row tiles)."""
    lo, hi = np.array([-1.0, -1.0, -1.0], np.float32), np.array([1.0, 1.0, 1.0], np.float32)
    c = _cache(lo, hi, seed=11)
    n = 3000
    q = _queries(n, lo, hi, seed=12)
    rng = np.random.default_rng(13)
    t = rng.uniform(0.0, 2.0, (n, 3)).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.2).astype(np.int32)
    gc = pt.Cache(ctx, c)
    loss, g = gc.loss_grad(torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mask).cuda())
    ctx.check()
    wl, wg = O.Cache(c).loss_grad(q.astype(np.float64), t.astype(np.float64), mask=mask)
    g = g.cpu().numpy().astype(np.float64)
    assert abs(loss.item() - wl) <= 1e-5 * abs(wl)
    assert np.linalg.norm(g - wg) <= 1e-4 * np.linalg.norm(wg)
    assert np.abs(g - wg).max() <= 1e-4 * np.abs(wg).max()
    # the loss-only call updates nothing
    assert np.array_equal(gc.get_params(), pt.cache_flat(c))


@pytest.mark.parametrize("J,L,H,n", [(12, 5, 64, 3000), (4, 3, 64, 129), (12, 5, 64, (1 << 16) + 3)])
def test_bf16_cache_loss_grad_matches_rounding_model(pt, ctx, J, L, H, n):
    """Tensor-core training GEMMs of the cache: relative-L2 loss and gradient
    against the BF16 rounding model (pinned to the oracle on the CPU) to
    2e-3 per layer, and against the FP64 oracle to 5e-2; 20% of the rows
    masked; two calls are bit-identical."""
    import bf16_model as BM
    lo, hi = np.array([-1.0, -1.0, -1.0], np.float32), np.array([1.0, 1.0, 1.0], np.float32)
    c = I.cache_init(lo, hi, n_freq=J, hidden=H, n_hidden_layers=L, seed=21)
    rng = np.random.default_rng(22)
    for b in c.b:
        b[:] = rng.normal(0, 0.1, b.shape).astype(np.float32)
    q = _queries(n, lo, hi, seed=23)
    t = rng.uniform(0.0, 2.0, (n, 3)).astype(np.float32)
    mask = (rng.uniform(size=n) > 0.2).astype(np.int32)
    gc = pt.Cache(ctx, c)
    args = (torch.from_numpy(q).cuda(), torch.from_numpy(t).cuda(), torch.from_numpy(mask).cuda())
    loss, g = gc.loss_grad(*args, precision="bf16")
    loss2, g2 = gc.loss_grad(*args, precision="bf16")
    ctx.check()
    assert torch.equal(loss, loss2) and torch.equal(g, g2)
    g = g.cpu().numpy().astype(np.float64)
    ml, mg = BM.mlp_loss_grad(BM.cache_features(c, q), c.W, c.b, t, "rel_l2", mask=mask)
    assert abs(loss.item() - ml) <= 1e-4 * abs(ml)
    wl, wg = O.Cache(c).loss_grad(q.astype(np.float64), t.astype(np.float64), mask=mask)
    assert abs(loss.item() - wl) <= 1e-2 * abs(wl)
    p = 0
    for W, b in zip(c.W, c.b):
        for size in (W.size, b.size):
            a, m, w = g[p:p + size], mg[p:p + size], wg[p:p + size]
            assert np.linalg.norm(a - m) <= 2e-3 * np.linalg.norm(m), (p, np.linalg.norm(a - m) / np.linalg.norm(m))
            assert np.linalg.norm(a - w) <= 5e-2 * np.linalg.norm(w)
            p += size


def test_bf16_cache_training_frames(pt, ctx):
    """Online frames with tensor-core training GEMMs: bit-reproducible, and
    the per-frame losses stay within 5% of the FP32-trained run's."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = _cache(lo, hi, seed=41)
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    runs = {}
    for tp in ("fp32", "bf16", "bf16"):
        gc = pt.Cache(ctx, c)
        losses = []
        for frame in range(8):
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
            gc.train_frame(s, g, 64, 64, frame, n_train=8192, loss=loss, train_precision=tp)
            losses.append(loss.item())
        ctx.check()
        runs.setdefault(tp, []).append((np.array(losses), gc.get_params()))
    (l32, _), = runs["fp32"]
    (la, pa), (lb, pb) = runs["bf16"]
    assert np.array_equal(la, lb) and np.array_equal(pa, pb)
    assert np.all(np.isfinite(la))
    assert np.all(np.abs(la - l32) <= 5e-2 * np.abs(l32)), np.abs(la - l32) / np.abs(l32)


def _box_setup(pt, ctx):
    return I.make_scene("C1"), I.nif_init(seed=0)


def test_records_match_oracle(pt, ctx):
    """Vertex-2 records (x, wo, n, tp, radiance before the vertex, valid) and
    path radiance on the box scene with the NIF, per path."""
    sc, nif = _box_setup(pt, ctx)
    cfg = I.RenderCfg(64, 64, 2, 4, 0)
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    pixels = np.arange(0, 64 * 64, 3, dtype=np.int64)
    pix, slots, rec, ids = pt.render_cached(ctx, s, g, cfg, torch.from_numpy(pixels).cuda(), rec_vertex=2,
                                            want_slots=True, want_ids=True)
    ctx.check()
    n = len(pixels)
    P = np.tile(pixels, cfg.spp)
    S = np.repeat(np.arange(cfg.spp), n)
    L, orec, oids = O.trace_paths(O.Scene(sc), sc.camera, cfg.width, cfg.height, cfg.max_depth, cfg.seed, P, S,
                                  nif=O.Nif(nif), rec_vertex=2, want_ids=True)
    gids = ids.cpu().numpy().reshape(-1, cfg.max_depth)
    same = np.all(gids == oids, axis=1)
    assert same.mean() >= 0.999
    grec = rec.cpu().numpy().reshape(-1, 16)
    assert np.array_equal(grec[same, 15], orec[same, 15])
    v = same & (orec[:, 15] == 1.0)
    assert v.sum() > 0.3 * len(v)
    assert np.abs(grec[v, :3] - orec[v, :3]).max() <= 1e-4 * max(1.0, np.abs(orec[v, :3]).max())
    assert np.abs(grec[v, 3:9] - orec[v, 3:9]).max() <= 1e-4
    assert np.abs(grec[v, 9:15] - orec[v, 9:15]).max() <= 1e-4 * max(1.0, np.abs(orec[v, 9:15]).max())
    assert np.all(grec[~(orec[:, 15] == 1.0) & same] == 0.0)
    gL = slots.cpu().numpy().reshape(-1, 3)
    assert rel_rmse(gL[same], L[same]) <= 1e-4


def test_cached_render_matches_oracle(pt, ctx):
    """Paths end at vertex 2 into a random cache: per-path radiance vs the
    oracle's cached paths."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = _cache(lo, hi, seed=21, bias_std=0.5)
    cfg = I.RenderCfg(64, 64, 4, 4, 0)
    s, g, gc = pt.Scene(ctx, sc), pt.Nif(ctx, nif), pt.Cache(ctx, c)
    pix, slots, _, ids = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, want_slots=True,
                                          want_ids=True)
    ctx.check()
    n = cfg.width * cfg.height
    P = np.tile(np.arange(n), cfg.spp)
    S = np.repeat(np.arange(cfg.spp), n)
    L, _, oids = O.trace_paths(O.Scene(sc), sc.camera, cfg.width, cfg.height, cfg.max_depth, cfg.seed, P, S,
                               nif=O.Nif(nif), cache=O.Cache(c), cache_vertex=2, want_ids=True)
    gids = ids.cpu().numpy().reshape(-1, cfg.max_depth)
    same = np.all(gids == oids, axis=1)
    assert same.mean() >= 0.999
    assert np.all(gids[:, 2:] == -2)
    gL = slots.cpu().numpy().reshape(-1, 3)
    assert rel_rmse(gL[same], L[same]) <= 1e-4
    img = L.reshape(cfg.spp, n, 3).mean(0)
    assert rel_rmse(pix.cpu().numpy(), img) <= 1e-3


def test_cached_render_furnace_closed_form(pt, ctx):
    """Closed sphere of albedo a and emission 1 - a, constant cache c at
    vertex 2 (negative outputs clamp to 0): every path gives (1 - a) + a c."""
    a = 0.6
    sc = I.furnace_sphere_inside(a)
    lo, hi = I.scene_bounds(sc)
    c = I.cache_init(lo, hi)
    for W in c.W:
        W[:] = 0
    for b in c.b:
        b[:] = 0
    c.b[-1][:] = [0.25, 0.5, -1.0]
    cfg = I.RenderCfg(32, 32, 4, 6, 0)
    img, slots, _, _ = pt.render_cached(ctx, pt.Scene(ctx, sc), None, cfg, None, cache=pt.Cache(ctx, c),
                                        cache_vertex=2, want_slots=True)
    ctx.check()
    af, le = float(sc.mat[0, 0]), float(sc.mat[0, 5])
    want = np.array([le + af * 0.25, le + af * 0.5, le])
    assert np.abs(slots.cpu().numpy() - want).max() <= 1e-6


def test_train_cache_step(pt, ctx):
    """One pt_train_cache frame equals its parts: training pixels from
    Philox (seed, 2), records of the plain paths at vertex 2, targets (L -
    L_before) / tp, the relative-L2 gradient (itself checked against the
    oracle here on the same rows) and one Adam step."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = _cache(lo, hi, seed=31)
    W, H, n, frame, seed, depth = 64, 64, 4096, 3, 0, 6
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    gc = pt.Cache(ctx, c)
    w0 = gc.get_params()
    loss = torch.zeros(1, dtype=torch.float32, device="cuda")
    gc.train_frame(s, g, W, H, frame, n_train=n, max_depth=depth, rec_vertex=2, seed=seed, loss=loss)
    ctx.check()
    w1 = gc.get_params()
    # the same step from its parts
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n)
    ctr[:, 1] = frame
    pixels = (O.philox_batch(seed, 2, ctr)[:, 0] % (W * H)).astype(np.int64)
    cfg = I.RenderCfg(W, H, 1, depth, seed)
    _, slots, rec, _ = pt.render_cached(ctx, s, g, cfg, torch.from_numpy(pixels).cuda(), rec_vertex=2,
                                        want_slots=True, first_sample=TRAIN_SAMPLE_BASE + frame)
    ctx.check()
    rec = rec.cpu().numpy().reshape(n, 16)
    Lp = slots.cpu().numpy().reshape(n, 3)
    tp = rec[:, 9:12]
    mask = ((rec[:, 15] != 0) & np.all(tp > 0, axis=1)).astype(np.int32)
    tgt = np.where(mask[:, None] == 1, (Lp - rec[:, 12:15]) / np.where(tp > 0, tp, 1), 0).astype(np.float32)
    assert mask.mean() > 0.3
    gcopy = pt.Cache(ctx, c)
    l2, grad = gcopy.loss_grad(torch.from_numpy(np.ascontiguousarray(rec[:, :9])).cuda(), torch.from_numpy(tgt).cuda(),
                               torch.from_numpy(mask).cuda())
    ctx.check()
    assert abs(l2.item() - loss.item()) <= 1e-6 * abs(l2.item())
    grad = grad.cpu().numpy()
    # gradient vs the oracle on these rows
    wl, wg = O.Cache(c).loss_grad(rec[:, :9].astype(np.float64), tgt.astype(np.float64), mask=mask)
    assert abs(l2.item() - wl) <= 1e-4 * abs(wl)
    assert np.linalg.norm(grad - wg) <= 1e-4 * np.linalg.norm(wg)
    # Adam, first step with bias correction
    lr, b1, b2, eps = 1e-2, 0.9, 0.999, 1e-7
    m = (1 - b1) * grad.astype(np.float64)
    v = (1 - b2) * grad.astype(np.float64) ** 2
    want = w0 - lr * (m / (1 - b1)) / (np.sqrt(v / (1 - b2)) + eps)
    assert np.abs(w1 - want).max() <= 1e-6 * max(1.0, np.abs(w0).max()) + 1e-5 * lr
    # targets of matched paths agree with the oracle's records
    S = np.full(n, TRAIN_SAMPLE_BASE + frame, np.int64)
    L, orec, _ = O.trace_paths(O.Scene(sc), sc.camera, W, H, depth, seed, pixels, S, nif=O.Nif(nif), rec_vertex=2)
    ok = (orec[:, 15] == 1) & (mask == 1)
    otgt = (L[ok] - orec[ok, 12:15]) / orec[ok, 9:12]
    close = np.abs(tgt[ok] - otgt) <= 1e-3 * np.maximum(1.0, np.abs(otgt))
    assert close.mean() >= 0.995


def test_trained_cache_reduces_bias(pt, ctx):
    """What training buys: on the box scene, a render that ends every path at
    vertex 2 in the cache is far closer to the plain full-depth render after
    100 online frames than with the random-init cache, and the relative-L2
    loss stays finite throughout."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = I.cache_init(lo, hi, seed=5)
    s, g, gc = pt.Scene(ctx, sc), pt.Nif(ctx, nif), pt.Cache(ctx, c)
    W = H = 64
    depth = 6
    ref = pt.render(ctx, s, g, I.RenderCfg(W, H, 4096, depth, 1)).double()
    hi_spp = I.RenderCfg(W, H, 1024, depth, 2)
    before = pt.render_cached(ctx, s, g, hi_spp, None, cache=gc, cache_vertex=2)[0].double()
    losses = []
    for f in range(100):
        loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        gc.train_frame(s, g, W, H, f, n_train=1 << 14, max_depth=depth, loss=loss)
        losses.append(loss)
    after = pt.render_cached(ctx, s, g, hi_spp, None, cache=gc, cache_vertex=2)[0].double()
    ctx.check()
    losses = np.array([x.item() for x in losses])
    assert np.all(np.isfinite(losses))
    r = ref.reshape(-1, 3)
    e0 = float(torch.sqrt(((before - r) ** 2).sum() / (r ** 2).sum()))
    e1 = float(torch.sqrt(((after - r) ** 2).sum() / (r ** 2).sum()))
    print(f"cache bias: untrained {e0:.4f}, trained {e1:.4f}; loss first {losses[:5].mean():.3f} "
          f"last {losses[-10:].mean():.3f}")
    assert e1 < 0.25 * e0, (e0, e1)
    assert e1 < 0.05, (e0, e1)


def test_cache_argument_errors(pt, ctx):
    lo, hi = [0, 0, 0], [1, 1, 1]
    c = I.cache_init(lo, hi, hidden=32)
    with pytest.raises(pt.PTError):
        pt.Cache(ctx, c)
    c = I.cache_init([0, 0, 0], [1, 1, 1])
    c.hi = np.array([1, 0, 1], np.float32)
    with pytest.raises(pt.PTError):
        pt.Cache(ctx, c)
    sc = I.make_scene("C1")
    c = I.cache_init(*I.scene_bounds(sc))
    gc = pt.Cache(ctx, c)
    cfg = I.RenderCfg(8, 8, 1, 4, 0)
    s = pt.Scene(ctx, sc)
    g = pt.Nif(ctx, I.nif_init(seed=0))
    with pytest.raises(pt.PTError):
        pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=1)
    with pytest.raises(pt.PTError):
        pt.render_cached(ctx, s, g, cfg, None, cache=None, cache_vertex=2)
    ctx.check()


def test_cached_render_chunking_is_invisible(pt, ctx):
    """Chunks of whole samples change nothing: the cache queue and records are
    rebuilt per chunk, so a render in one-sample chunks equals the one-chunk
    render bit for bit, in FP32 and in BF16."""
    sc, nif = _box_setup(pt, ctx)
    lo, hi = I.scene_bounds(sc)
    c = _cache(lo, hi, seed=51, bias_std=0.5)
    cfg = I.RenderCfg(48, 40, 5, 4, 0)
    s, g, gc = pt.Scene(ctx, sc), pt.Nif(ctx, I.nif_init(colour="yuv")), pt.Cache(ctx, c)
    for prec in ("fp32", "bf16"):
        one = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, rec_vertex=2, precision=prec,
                               want_slots=True)
        many = pt.render_cached(ctx, s, g, cfg, None, cache=gc, cache_vertex=2, rec_vertex=2, precision=prec,
                                want_slots=True, chunk_slots=48 * 40)
        ctx.check()
        assert torch.equal(one[1], many[1]) and torch.equal(one[2], many[2])
        assert torch.allclose(one[0], many[0], rtol=1e-6, atol=0)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_pt_render_with_cache_equals_render_cached(pt, ctx, precision):
    """A full cached image from one pt_render call (cache and cfg cache_vertex)
    is bit for bit pt_render_cached over every pixel: C5 at 1024x1024, 4 spp,
    cache at vertex 2."""
    sc, nif, cfg = I.make_scene("C5"), I.nif_init(colour="yuv"), I.CONFIGS["C5"]["cfg"]
    lo, hi = I.scene_bounds(sc)
    s, g, c = pt.Scene(ctx, sc), pt.Nif(ctx, nif), pt.Cache(ctx, _cache(lo, hi))
    img = pt.render(ctx, s, g, cfg, precision, cache=c, cache_vertex=2)
    ref = pt.render_cached(ctx, s, g, cfg, None, cache=c, cache_vertex=2, precision=precision)[0]
    ctx.check()
    assert torch.equal(img.reshape(-1, 3), ref)
    plain = pt.render(ctx, s, g, cfg, precision)
    ctx.check()
    assert not torch.equal(plain, img)        # the cache did end the paths


def test_pt_render_cache_arguments(pt, ctx):
    import ctypes
    sc = I.make_scene("C1")
    lo, hi = I.scene_bounds(sc)
    s, g, c = pt.Scene(ctx, sc), pt.Nif(ctx, I.nif_init()), pt.Cache(ctx, _cache(lo, hi))
    cfg = I.RenderCfg(8, 8, 1, 3)
    out = torch.empty((8, 8, 3), device="cuda")
    for cache, cv in ((c, 0), (c, 1), (None, 2)):
        k = pt.make_cfg(cfg, cache_vertex=cv)
        st = pt.lib().pt_render(ctx.h, s.h, g.h, cache.h if cache is not None else None, ctypes.byref(k),
                                pt._dptr(out), None)
        assert st == pt.PT_EINVAL, (cache, cv)
    k = pt.make_cfg(cfg, cache_vertex=2)       # render_pixels has no cache
    st = pt.lib().pt_render_pixels(ctx.h, s.h, g.h, ctypes.byref(k), 0, None, pt._dptr(out), None, None, None)
    assert st == pt.PT_EINVAL
    ctx.check()
