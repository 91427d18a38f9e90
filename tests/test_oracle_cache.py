"""Pins of the oracle's neural radiance cache (CPU only): encoding and
forward pass by closed-form wiring, the relative-L2 gradient by finite
differences on its fixed-denominator form and a closed form for the output
bias, suffix-radiance records and cached rendering in the white furnace."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I


def _zero(c):
    z = c.copy()
    for W in z.W:
        W[:] = 0
    for b in z.b:
        b[:] = 0
    return z


def _queries(n, rng, lo=-1.0, hi=1.0):
    x = rng.uniform(lo, hi, (n, 3))
    d = rng.normal(0, 1, (n, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    nn = rng.normal(0, 1, (n, 3))
    nn /= np.linalg.norm(nn, axis=1, keepdims=True)
    return np.concatenate([x, d, nn], 1)


def test_cache_zero_weights_return_output_bias():
    c = _zero(I.cache_init([-1, -1, -1], [1, 1, 1], n_freq=4, hidden=8, n_hidden_layers=2))
    c.b[-1][:] = [0.5, 1.5, -2.0]
    out = O.Cache(c).forward(_queries(10, np.random.default_rng(0)))
    assert np.allclose(out, [0.5, 1.5, -2.0], atol=0)


def test_cache_encoding_by_wiring():
    """relu(x) - relu(-x) = x passes single features: the sine of frequency 3
    of normalised y to channel 0, the direction's z to channel 1, the
    normal's x to channel 2."""
    J = 5
    c = _zero(I.cache_init([-2, 0, 1], [2, 4, 3], n_freq=J, hidden=8, n_hidden_layers=2))
    feat = [1 * 2 * J + 3, 6 * J + 2, 6 * J + 3]   # sin(2^3 pi p_y), dir z, normal x
    for ch, f in enumerate(feat):
        c.W[0][2 * ch, f] = 1.0
        c.W[0][2 * ch + 1, f] = -1.0
        c.W[1][2 * ch, 2 * ch] = 1.0
        c.W[1][2 * ch + 1, 2 * ch + 1] = 1.0
        c.W[2][ch, 2 * ch] = 1.0
        c.W[2][ch, 2 * ch + 1] = -1.0
    q = _queries(40, np.random.default_rng(1))
    q[:, :3] = np.random.default_rng(2).uniform([-2, 0, 1], [2, 4, 3], (40, 3))
    out = O.Cache(c).forward(q)
    py = (q[:, 1] - 0.0) / 4.0
    assert np.allclose(out[:, 0], np.sin(8 * math.pi * py), atol=1e-12)
    assert np.allclose(out[:, 1], q[:, 5], atol=1e-15)
    assert np.allclose(out[:, 2], q[:, 6], atol=1e-15)


def test_relative_l2_gradient_finite_differences():
    c = I.cache_init([-1, -1, -1], [1, 1, 1], n_freq=3, hidden=10, n_hidden_layers=3, seed=4)
    rng = np.random.default_rng(5)
    for b in c.b:
        b[:] = rng.normal(0, 0.2, b.shape)
    oc = O.Cache(c)
    q = _queries(6, rng)
    t = rng.uniform(0, 2, (6, 3))
    denom = rng.uniform(0.5, 2.0, (6, 3))
    mask = np.array([1, 1, 0, 1, 1, 1], np.int32)
    loss, g = oc.loss_grad(q, t, denom=denom, mask=mask)
    w0 = oc.get_params()
    h = 1e-6
    idx = list(range(0, len(w0), max(1, len(w0) // 150))) + [len(w0) - 1]
    for i in idx:
        wp, wm = w0.copy(), w0.copy()
        wp[i] += h
        wm[i] -= h
        oc.set_params(wp)
        lp, _ = oc.loss_grad(q, t, denom=denom, mask=mask)
        oc.set_params(wm)
        lm, _ = oc.loss_grad(q, t, denom=denom, mask=mask)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.abs(g).max()) + 1e-12, (i, fd, g[i])
    oc.set_params(w0)


def test_relative_l2_output_bias_closed_form():
    """d loss / d b_out = sum_s 2 (y - t) / (y^2 + 0.01) / (3 n) with y held
    constant in the denominator."""
    c = I.cache_init([-1, -1, -1], [1, 1, 1], n_freq=2, hidden=6, n_hidden_layers=2, seed=6)
    oc = O.Cache(c)
    q = _queries(5, np.random.default_rng(7))
    y = oc.forward(q)
    t = y + np.array([0.1, -0.2, 0.3])
    loss, g = oc.loss_grad(q, t)
    want = (2 * (y - t) / (y ** 2 + 0.01)).sum(0) / 15.0
    assert np.allclose(g[-3:], want, rtol=1e-12)
    assert abs(loss - (((y - t) ** 2) / (y ** 2 + 0.01)).sum() / 15.0) < 1e-14


def test_records_give_suffix_radiance_in_furnace():
    """Closed sphere, albedo a, emission 1 - a, depth D: the radiance a path
    gathers from vertex k onwards divided by the throughput reaching it is
    1 - a^(D - k + 1)."""
    a, D, k = 0.6, 6, 2
    sc = I.furnace_sphere_inside(a)
    os_ = O.Scene(sc)
    n = 50
    L, rec, _ = O.trace_paths(os_, sc.camera, 16, 16, D, 0, np.arange(n) % 256, np.arange(n) // 256,
                              rec_vertex=k)
    af, le = float(sc.mat[0, 0]), float(sc.mat[0, 5])
    assert np.all(rec[:, 15] == 1.0)
    tgt = (L - rec[:, 12:15]) / rec[:, 9:12]
    want = le * sum(af ** m for m in range(D - k + 1))
    assert np.allclose(tgt, want, atol=1e-13)
    assert np.allclose(rec[:, 9:12], af ** (k - 1), atol=1e-15)


def test_cached_render_closed_form():
    """A constant cache c at vertex 2 in the closed furnace: L = (1 - a) + a c."""
    a = 0.6
    sc = I.furnace_sphere_inside(a)
    lo, hi = I.scene_bounds(sc)
    c = _zero(I.cache_init(lo, hi, n_freq=3, hidden=8, n_hidden_layers=2))
    c.b[-1][:] = [0.25, 0.5, -1.0]   # negative outputs are clamped to zero
    oc = O.Cache(c)
    L, _, ids = O.trace_paths(O.Scene(sc), sc.camera, 8, 8, 6, 0, np.arange(64), np.zeros(64, np.int64), cache=oc,
                              cache_vertex=2, want_ids=True)
    af, le = float(sc.mat[0, 0]), float(sc.mat[0, 5])
    want = np.array([le + af * 0.25, le + af * 0.5, le])
    assert np.allclose(L, want, atol=1e-13)
    assert np.all(ids[:, 2:] == -2)
