"""The skip-concatenated NIF (Section 3.2: one hidden layer's output joined
with the Fourier features before the next layer) through the C ABI against
the FP64 oracle: evaluation, loss and gradient, Adam steps, renders and
checkpoints; the precisions without a kernel for it refuse it."""
import os

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# (n_freq, hidden, hidden layers, skip layer): the paper's network (20 frequencies, 4 x 128, joined after
# layer 2), the same with 32 frequencies, and small shapes with the join early and late
SHAPES = [(20, 128, 4, 2), (32, 128, 4, 2), (5, 12, 2, 1), (3, 9, 5, 4)]


@pytest.fixture(scope="module")
def pt():
    from paper_2305_20061_gb300 import build
    build.build()
    from paper_2305_20061_gb300 import pt as _pt
    return _pt


@pytest.fixture(scope="module")
def ctx(pt):
    return pt.Context(0)


def _nif(F, H, L, S, seed=0):
    nif = I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L, colour="yuv", seed=seed, skip_after=S)
    rng = np.random.default_rng(seed + 11)
    for b in nif.b:
        b[:] = rng.normal(0, 0.05, b.shape).astype(np.float32)
    return nif


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))


def test_paper_network_size(pt, ctx):
    """20 frequencies, four hidden layers of 128 joined after the second:
    50,011 trainable parameters (97.7 KiB in FP16); the device's flat layout
    adds the 2F frequencies and the 3x3 colour matrix."""
    g = pt.Nif(ctx, I.nif_init(n_freq=20, hidden=128, n_hidden_layers=4, skip_after=I.paper_skip_layer(4)))
    assert I.paper_skip_layer(4) == 2 and g.param_count == 50011 + 2 * 20 + 9


@pytest.mark.parametrize("shape", SHAPES)
def test_eval_matches_oracle(pt, ctx, shape):
    """FP32 evaluation within 1e-5 relative per channel of the FP64 oracle
    on the same float32 (u, v): several 128-row tiles and a ragged tail."""
    nif = _nif(*shape)
    g = pt.Nif(ctx, nif)
    uv = I.uniform_uv(128 * 37 + 41, seed=5)
    uv[:3] = [[0, 0], [0.999999, 0.999999], [0.5, 0.5]]
    rgb = g.eval(torch.from_numpy(uv).cuda()).cpu().numpy().astype(np.float64)
    ctx.check()
    ref, _ = O.Nif(nif).forward(uv.astype(np.float64))
    rel = np.abs(rgb - ref) / np.abs(ref)
    assert rel.max() <= 1e-5, rel.max()


def test_join_changes_the_output(pt, ctx):
    """Zeroing the weights that read the joined features changes the
    device's output (the features really enter after the skip layer) and
    still matches the oracle."""
    nif = _nif(20, 128, 4, 2)
    uv = I.uniform_uv(2000, seed=9)
    a = pt.Nif(ctx, nif).eval(torch.from_numpy(uv).cuda()).cpu().numpy()
    cut = nif.copy()
    cut.W[2][:, 128 - 40:] = 0.0
    b = pt.Nif(ctx, cut).eval(torch.from_numpy(uv).cuda()).cpu().numpy()
    ctx.check()
    ref, _ = O.Nif(cut).forward(uv.astype(np.float64))
    assert _rel(b, ref) <= 1e-5
    assert _rel(a, b) > 1e-3


@pytest.mark.parametrize("delta", [10.0, 1e-3])
@pytest.mark.parametrize("shape", SHAPES)
def test_loss_and_gradient_match_oracle(pt, ctx, shape, delta):
    nif = _nif(*shape)
    g = pt.Nif(ctx, nif)
    n = 128 * 37 + 5
    uv = I.uniform_uv(n, seed=3)
    _, z = O.Nif(nif).forward(uv.astype(np.float64))
    target = (z + np.random.default_rng(4).normal(0, 0.5, z.shape)).astype(np.float32)
    loss, grad = g.loss_grad(torch.from_numpy(uv).cuda(), torch.from_numpy(target).cuda(), delta)
    ctx.check()
    ref_loss, ref_grad = O.Nif(nif).loss_grad(uv.astype(np.float64), target.astype(np.float64), delta)
    assert abs(float(loss.item()) - ref_loss) <= 1e-5 * abs(ref_loss)
    got = grad.cpu().numpy().astype(np.float64)
    p = 0
    for W, b in zip(nif.W, nif.b):
        for size in (W.size, b.size):
            assert _rel(got[p:p + size], ref_grad[p:p + size]) <= 1e-4, (p, size)
            p += size
    assert p == got.size


def test_adam_steps_match_oracle(pt, ctx):
    """Three Adam steps of the paper's network on the procedural sky from the
    same Philox samples: per-step losses and the updated weights agree."""
    nif = _nif(20, 128, 4, 2)
    sky = I.procedural_sky(128, 64)
    g = pt.Nif(ctx, nif)
    steps, batch, lr = 3, 512, 1e-3
    losses = g.train(torch.from_numpy(sky).cuda(), steps=steps, batch=batch, lr=lr, seed=5).cpu().numpy()
    ctx.check()
    on = O.Nif(nif)
    ref_losses = on.train(sky, seed=5, steps=steps, batch=batch, lr=lr)
    assert np.allclose(losses, ref_losses, rtol=1e-4), (losses, ref_losses)
    got = g.get_params().astype(np.float64)[2 * nif.n_freq:-9]
    ref = on.get_trainable()
    # every weight moved by about lr per step; agreement to a small fraction of one step
    assert np.abs(got - ref).max() <= 0.05 * lr, np.abs(got - ref).max()
    # the FP32 layout used by evaluation follows the trained weights
    trained = pt.nif_from_flat(20, 128, 4, g.get_params(), 2)
    uv = I.uniform_uv(1000, seed=8)
    rgb = g.eval(torch.from_numpy(uv).cuda()).cpu().numpy()
    ref_rgb, _ = O.Nif(trained).forward(uv.astype(np.float64))
    assert _rel(rgb, ref_rgb) <= 1e-5


def test_training_lowers_the_loss(pt, ctx):
    nif = _nif(20, 128, 4, 2)
    g = pt.Nif(ctx, nif)
    losses = g.train(torch.from_numpy(I.procedural_sky(256, 128)).cuda(), steps=200, batch=4096, lr=3e-3,
                     seed=1).cpu().numpy()
    ctx.check()
    assert np.all(np.isfinite(losses)) and losses[-20:].mean() < 0.5 * losses[:5].mean(), losses[[0, -1]]


def test_checkpoint_round_trip(pt, ctx, tmp_path):
    nif = _nif(20, 128, 4, 2)
    g = pt.Nif(ctx, nif)
    g.train(torch.from_numpy(I.procedural_sky(128, 64)).cuda(), steps=2, batch=256, lr=1e-3)
    path = os.path.join(tmp_path, "skip.ptck")
    g.save(path)
    ctx.check()
    assert pt.checkpoint_info(path)["dims"][:4] == [20, 128, 4, 2]
    h = pt.Nif.load(ctx, path)
    assert h.src.skip_after == 2 and np.array_equal(h.get_params(), g.get_params())
    uv = torch.from_numpy(I.uniform_uv(3000, seed=2)).cuda()
    assert torch.equal(h.eval(uv), g.eval(uv))
    # training resumes from the stored Adam state identically
    sky = torch.from_numpy(I.procedural_sky(128, 64)).cuda()
    a = g.train(sky, steps=2, batch=256, lr=1e-3, seed=7)
    b = h.train(sky, steps=2, batch=256, lr=1e-3, seed=7)
    ctx.check()
    assert torch.equal(a, b) and np.array_equal(h.get_params(), g.get_params())


def test_render_with_the_skip_network_matches_oracle(pt, ctx):
    """The box scene (C1's 64x64, 8 spp, depth 4) lit by the skip network:
    per-path radiance of paths with the same hit sequence within 1e-3."""
    from parity_helpers import rel_rmse
    cfg = I.CONFIGS["C1"]["cfg"]
    sc, nif = I.box_scene(), _nif(20, 128, 4, 2)
    img, slots, ids = pt.render_pixels(ctx, pt.Scene(ctx, sc), pt.Nif(ctx, nif), cfg, None, want_slots=True,
                                       want_ids=True)
    ctx.check()
    r = O.render(O.Scene(sc), cfg, O.Nif(nif), want_slots=True, want_ids=True)
    gslots = slots.cpu().numpy().transpose(1, 0, 2)
    same = ~np.any(ids.cpu().numpy().transpose(1, 0, 2) != r["ids"], axis=2)
    assert same.mean() >= 1 - 1e-3
    assert rel_rmse(gslots[same], r["slots"][same]) <= 1e-3
    assert rel_rmse(img.cpu().numpy(), r["image"]) <= 1e-3


def test_precisions_without_a_kernel_refuse(pt, ctx):
    """The paper's network has a BF16 tensor-core kernel (tested with the
    other tensor-core shapes); FP8 evaluation, BF16 training and other skip
    shapes in BF16 are refused."""
    nif = _nif(20, 128, 4, 2)
    g = pt.Nif(ctx, nif)
    uv = torch.from_numpy(I.uniform_uv(100, seed=1)).cuda()
    g.eval(uv, precision="bf16")
    with pytest.raises(pt.PTError) as e:
        g.eval(uv, precision="fp8")
    assert e.value.status == pt.PT_EUNSUPPORTED
    with pytest.raises(pt.PTError) as e:
        g.train(torch.from_numpy(I.procedural_sky(64, 32)).cuda(), steps=1, batch=128, precision="bf16")
    assert e.value.status == pt.PT_EUNSUPPORTED
    other = pt.Nif(ctx, _nif(32, 128, 4, 2))
    with pytest.raises(pt.PTError) as e:
        other.eval(uv, precision="bf16")
    assert e.value.status == pt.PT_EUNSUPPORTED
    with pytest.raises(pt.PTError) as e:
        pt.render(ctx, pt.Scene(ctx, I.box_scene()), other, I.RenderCfg(8, 8, 1, 2), "bf16")
    assert e.value.status == pt.PT_EUNSUPPORTED
    ctx.check()


def test_load_rejects_bad_skip(pt, ctx):
    for F, H, L, S in [(20, 128, 4, 4), (20, 40, 4, 2), (20, 128, 4, -1)]:
        nif = I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L)
        nif.skip_after = S
        with pytest.raises(pt.PTError) as e:
            pt.Nif(ctx, nif)
        assert e.value.status == pt.PT_EINVAL
