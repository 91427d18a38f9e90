"""Pins of the BF16 training rounding model (tests/bf16_model.py) on the
CPU: BF16 rounding on values whose nearest BF16 is known, and, with rounding
off, the model's backpropagation against the FP64 oracle's gradient of the
NIF Huber loss (Section 3.2.1) and of the radiance cache's relative L2 loss."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

import bf16_model as BM


def test_bf16_rounding_known_values():
    # ties go to the even mantissa; just above a tie rounds up; 2^100 (1 + 2^-7 + 2^-9) is below the tie
    x = np.array([1.0, 1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, 1.0 + 2.0 ** -8 + 2.0 ** -20, -2.5,
                  2.0 ** 100 * (1 + 2.0 ** -7 + 2.0 ** -9), 0.0, 2.0 ** -130], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2.0 ** -6, 1.0 + 2.0 ** -7, -2.5, 2.0 ** 100 * (1 + 2.0 ** -7), 0.0,
                     2.0 ** -130], np.float32)
    assert np.array_equal(BM.bf16(x), want)


def _nif(F, H, L, seed):
    nif = I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L, colour="yuv", seed=seed)
    rng = np.random.default_rng(seed + 1)
    for b in nif.b:
        b[:] = rng.normal(0, 0.05, b.shape).astype(np.float32)
    return nif


@pytest.mark.parametrize("delta", [10.0, 1e-3])
@pytest.mark.parametrize("shape", [(8, 32, 3), (5, 12, 2)])
def test_model_without_rounding_is_the_oracle_nif_gradient(delta, shape):
    nif = _nif(*shape, seed=2)
    n = 300
    uv = I.uniform_uv(n, seed=7)
    _, z = O.Nif(nif).forward(uv.astype(np.float64))
    target = z + np.random.default_rng(8).normal(0, 0.5, z.shape)
    ref_loss, ref_grad = O.Nif(nif).loss_grad(uv.astype(np.float64), target, delta)
    X0 = BM.nif_features(nif.B, uv, fp32=False)
    loss, grad = BM.mlp_loss_grad(X0, nif.W, nif.b, target, "huber", M=nif.M, delta=delta, rounding=False)
    assert abs(loss - ref_loss) <= 1e-9 * abs(ref_loss)
    assert np.linalg.norm(grad - ref_grad) <= 1e-9 * np.linalg.norm(ref_grad)


def test_model_without_rounding_is_the_oracle_cache_gradient():
    lo, hi = np.array([-1.0, -2.0, 0.5], np.float32), np.array([1.0, 0.0, 3.0], np.float32)
    c = I.cache_init(lo, hi, n_freq=4, hidden=16, n_hidden_layers=3, seed=5)
    rng = np.random.default_rng(6)
    for b in c.b:
        b[:] = rng.normal(0, 0.1, b.shape).astype(np.float32)
    n = 257
    x = rng.uniform(lo, hi, (n, 3))
    d = rng.normal(0, 1, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    nn = rng.normal(0, 1, (n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    q = np.concatenate([x, d, nn], 1).astype(np.float32).astype(np.float64)
    t = rng.uniform(0.0, 2.0, (n, 3))
    mask = (rng.uniform(size=n) > 0.3).astype(np.int32)
    ref_loss, ref_grad = O.Cache(c).loss_grad(q, t, mask=mask)
    X0 = BM.cache_features(c, q, fp32=False)
    loss, grad = BM.mlp_loss_grad(X0, c.W, c.b, t, "rel_l2", mask=mask, rounding=False)
    assert abs(loss - ref_loss) <= 1e-9 * abs(ref_loss)
    assert np.linalg.norm(grad - ref_grad) <= 1e-9 * np.linalg.norm(ref_grad)


def test_rounding_moves_the_gradient_by_bf16_sized_amounts():
    """With rounding on, the gradient differs from FP64 by about the BF16
    unit roundoff (2^-9) times a modest factor, not by zero or by O(1)."""
    nif = _nif(16, 64, 3, seed=4)
    uv = I.uniform_uv(512, seed=9)
    _, z = O.Nif(nif).forward(uv.astype(np.float64))
    target = z + np.random.default_rng(10).normal(0, 0.5, z.shape)
    X0 = BM.nif_features(nif.B, uv)
    _, g64 = BM.mlp_loss_grad(X0, nif.W, nif.b, target, "huber", M=nif.M, delta=1e-3, rounding=False)
    _, g16 = BM.mlp_loss_grad(X0, nif.W, nif.b, target, "huber", M=nif.M, delta=1e-3, rounding=True)
    rel = np.linalg.norm(g16 - g64) / np.linalg.norm(g64)
    assert 2.0 ** -14 < rel < 2.0 ** -3, rel
