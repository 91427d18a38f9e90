"""Checkpoints through the C ABI: a saved NIF or radiance cache loads back
with identical weights and training state, and training resumed from the
file continues the run bit-exactly (the same losses and weights as the run
that never stopped), in both training precisions.  Wrong-kind and damaged
files are refused."""
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


def test_untrained_nif_round_trip(pt, ctx, tmp_path):
    nif = I.nif_init(colour="yuv", seed=3)
    g = pt.Nif(ctx, nif)
    path = str(tmp_path / "nif.ckpt")
    g.save(path)
    info = pt.checkpoint_info(path)
    assert info["kind"] == "nif" and info["dims"][:3] == [64, 128, 3] and info["n_adam"] == 0
    h = pt.Nif.load(ctx, path)
    assert np.array_equal(h.get_params(), g.get_params())
    assert np.array_equal(h.get_params(), O.nif_flat(nif))
    uv = torch.from_numpy(I.uniform_uv(4096, seed=1)).cuda()
    for prec in ("fp32", "bf16"):
        assert torch.equal(g.eval(uv, prec), h.eval(uv, prec))
    ctx.check()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_nif_training_resumes_bit_exactly(pt, ctx, tmp_path, precision):
    nif = I.nif_init(colour="yuv", seed=4)
    sky = torch.from_numpy(I.procedural_sky(128, 64)).cuda()
    kw = dict(batch=2048, lr=1e-2, seed=6, precision=precision)
    straight = pt.Nif(ctx, nif)
    l_all = straight.train(sky, steps=6, **kw).cpu().numpy()
    first = pt.Nif(ctx, nif)
    l_a = first.train(sky, steps=3, **kw).cpu().numpy()
    path = str(tmp_path / f"nif_{precision}.ckpt")
    first.save(path)
    info = pt.checkpoint_info(path)
    assert info["adam_t"] == 3 and info["n_adam"] == first.param_count - 2 * 64 - 9
    resumed = pt.Nif.load(ctx, path)
    l_b = resumed.train(sky, steps=3, **kw).cpu().numpy()
    ctx.check()
    assert np.array_equal(np.concatenate([l_a, l_b]), l_all)
    assert np.array_equal(resumed.get_params(), straight.get_params())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_cache_training_resumes_bit_exactly(pt, ctx, tmp_path, precision):
    sc = I.box_scene()
    nif = I.nif_init(colour="yuv", seed=7)
    s, g = pt.Scene(ctx, sc), pt.Nif(ctx, nif)
    lo, hi = I.scene_bounds(sc)
    cache = I.cache_init(lo, hi, seed=8)

    def frames(c, f0, n):
        out = []
        for f in range(f0, f0 + n):
            loss = torch.zeros(1, dtype=torch.float32, device="cuda")
            c.train_frame(s, g, 64, 64, f, n_train=4096, loss=loss, train_precision=precision)
            out.append(loss.item())
        return out

    straight = pt.Cache(ctx, cache)
    l_all = frames(straight, 0, 4)
    first = pt.Cache(ctx, cache)
    l_a = frames(first, 0, 2)
    path = str(tmp_path / f"cache_{precision}.ckpt")
    first.save(path)
    info = pt.checkpoint_info(path)
    assert info["kind"] == "cache" and info["adam_t"] == 2 and info["n_adam"] == first.param_count
    assert np.allclose(info["lo"], lo) and np.allclose(info["hi"], hi)
    resumed = pt.Cache.load(ctx, path)
    assert np.array_equal(resumed.src.lo, np.asarray(lo, np.float32))
    l_b = frames(resumed, 2, 2)
    ctx.check()
    assert l_a + l_b == l_all
    assert np.array_equal(resumed.get_params(), straight.get_params())


def test_wrong_kind_and_damaged_files(pt, ctx, tmp_path):
    g = pt.Nif(ctx, I.nif_init(seed=9))
    path = tmp_path / "n.ckpt"
    g.save(str(path))
    with pytest.raises(pt.PTError) as e:
        pt.Cache.load(ctx, str(path))
    assert e.value.status == pt.PT_EINVAL
    data = bytearray(path.read_bytes())
    data[200] ^= 0x40
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(bytes(data))
    with pytest.raises(pt.PTError) as e:
        pt.Nif.load(ctx, str(bad))
    assert e.value.status == pt.PT_EIO
    with pytest.raises(pt.PTError) as e:
        g.save(str(tmp_path / "no_such_dir" / "x.ckpt"))
    assert e.value.status == pt.PT_EIO
    ctx.check()
