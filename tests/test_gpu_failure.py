"""Failure detection without a GPU fault: a bounded device wait that nothing
satisfies gives up and reports PT_ERR_TIMEOUT; non-finite radiance sets
PT_ERR_NONFINITE; an allocation the device cannot satisfy returns PT_ENOMEM.
After each, the error word is clear again and the same context renders a
correct frame (the GPU stays usable)."""
import time

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


def _still_usable(pt, ctx):
    """the furnace-outside scene renders its closed-form values: the albedo where the sphere covers the
    pixel (centre), 1 where it does not (corner), in between only on the silhouette"""
    sc = I.furnace_sphere_outside(albedo=0.5)
    img = pt.render(ctx, pt.Scene(ctx, sc), None, I.RenderCfg(16, 16, 2, 3)).cpu().numpy()
    assert ctx.check() == 0
    assert np.allclose(img[8, 8], 0.5, rtol=1e-6) and np.allclose(img[0, 0], 1.0, rtol=1e-6)
    assert img.min() >= 0.5 - 1e-6 and img.max() <= 1.0 + 1e-6


@pytest.mark.parametrize("seconds", [0.02, 0.2])
def test_device_wait_gives_up_and_reports(pt, ctx, seconds):
    t0 = time.perf_counter()
    waited = ctx.selftest_wait_timeout(seconds)
    elapsed = time.perf_counter() - t0
    assert seconds <= waited < seconds + 0.5, waited
    assert elapsed < seconds + 5.0
    with pytest.raises(pt.PTError) as e:
        ctx.check()
    assert e.value.status == pt.PT_EDEVICE and e.value.bits & 0x8   # PT_ERR_TIMEOUT
    assert ctx.check() == 0                                           # read and cleared
    _still_usable(pt, ctx)


def test_device_error_bits_reads_without_clearing(pt, ctx):
    """pt_device_error_bits shows the word as it stands, as often as asked;
    pt_check then reports and clears it."""
    assert ctx.check() == 0
    assert pt.device_error_bits(ctx) == 0
    ctx.selftest_wait_timeout(0.02)
    assert pt.device_error_bits(ctx) == 0x8 and pt.device_error_bits(ctx) == 0x8
    with pytest.raises(pt.PTError) as e:
        ctx.check()
    assert e.value.bits == 0x8
    assert pt.device_error_bits(ctx) == 0
    assert pt.lib().pt_device_error_bits(None) == 0x80000000          # PT_ERR_UNREADABLE


def test_wait_selftest_arguments(pt, ctx):
    for bad in (0.0, -1.0, 3.0):
        with pytest.raises(pt.PTError) as e:
            ctx.selftest_wait_timeout(bad)
        assert e.value.status == pt.PT_EINVAL
    assert ctx.check() == 0


def test_nonfinite_radiance_is_flagged(pt, ctx):
    """An output bias of 200 overflows exp() in FP32: every escape's radiance
    is +inf, which the NIF kernels flag; FP32 and BF16 paths alike."""
    nif = I.nif_init(seed=2)
    nif.b[-1][:] = 200.0
    s = pt.Scene(ctx, I.box_scene())
    g = pt.Nif(ctx, nif)
    for prec in ("fp32", "bf16"):
        pt.render(ctx, s, g, I.RenderCfg(16, 16, 1, 2), prec)
        with pytest.raises(pt.PTError) as e:
            ctx.check()
        assert e.value.status == pt.PT_EDEVICE and e.value.bits & 0x4   # PT_ERR_NONFINITE
    _still_usable(pt, ctx)


def test_allocation_failure_returns_enomem(pt, ctx):
    """Training buffers for 2^36 samples (hundreds of TB) cannot be allocated:
    PT_ENOMEM, nothing trained, and a normal batch trains afterwards."""
    nif = I.nif_init(colour="yuv", seed=5)
    g = pt.Nif(ctx, nif)
    w0 = g.get_params()
    sky = torch.from_numpy(I.procedural_sky(64, 32)).cuda()
    with pytest.raises(pt.PTError) as e:
        g.train(sky, steps=1, batch=1 << 36)
    assert e.value.status == pt.PT_ENOMEM
    assert np.array_equal(g.get_params(), w0)
    losses = g.train(sky, steps=2, batch=1024).cpu().numpy()
    assert np.all(np.isfinite(losses))
    assert ctx.check() == 0
    _still_usable(pt, ctx)
