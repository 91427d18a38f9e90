"""Pins of the oracle's neural image field (forward, Huber-loss gradient,
Adam) and of its sky lookup, by closed-form constructions, finite
differences and textbook special cases (CPU only)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I


def _zero_like(nif):
    z = nif.copy()
    for W in z.W:
        W[:] = 0
    for b in z.b:
        b[:] = 0
    return z


def test_zero_frequencies_make_constant_features():
    """B = 0: every feature is sin 0 = 0 or cos 0 = 1, so the output does not
    depend on (u, v)."""
    nif = I.nif_init(n_freq=8, hidden=16, n_hidden_layers=2)
    nif.B[:] = 0
    o = O.Nif(nif)
    rgb, _ = o.forward(np.random.default_rng(0).uniform(0, 1, (20, 2)))
    assert np.allclose(rgb, rgb[0], rtol=0, atol=0)


def test_zero_weights_give_exp_of_colour_matrix_times_bias():
    nif = _zero_like(I.nif_init(n_freq=4, hidden=8, n_hidden_layers=3, colour="yuv"))
    nif.b[-1][:] = [0.3, -0.2, 0.1]
    nif.b[0][:] = 5.0  # hidden biases do not reach the output when the next weights are 0
    rgb, z = O.Nif(nif).forward([[0.3, 0.7]])
    M = nif.M.astype(np.float64)
    want = M @ nif.b[-1].astype(np.float64)
    assert np.allclose(z[0], want, atol=1e-15) and np.allclose(rgb[0], np.exp(want), rtol=1e-15)


def test_relu_pair_passes_a_single_fourier_feature():
    """relu(x) - relu(-x) = x: a network wired to pass feature i through
    gives exp(sin(2 pi (B_i0 u + B_i1 v))) in channel 0; with the cosine
    feature, channel 1; the colour matrix permutes channels."""
    F, H = 6, 8
    nif = _zero_like(I.nif_init(n_freq=F, hidden=H, n_hidden_layers=2))
    i_sin, i_cos = 2, F + 4  # sin of frequency 2, cos of frequency 4
    nif.W[0][0, i_sin] = 1.0
    nif.W[0][1, i_sin] = -1.0
    nif.W[0][2, i_cos] = 1.0
    nif.W[0][3, i_cos] = -1.0
    for j in range(4):
        nif.W[1][j, j] = 1.0
    nif.W[2][0, 0], nif.W[2][0, 1] = 1.0, -1.0
    nif.W[2][1, 2], nif.W[2][1, 3] = 1.0, -1.0
    nif.M[:] = [[0, 1, 0], [1, 0, 0], [0, 0, 1]]  # swap channels 0 and 1
    uv = np.random.default_rng(1).uniform(0, 1, (50, 2)).astype(np.float32).astype(np.float64)
    rgb, z = O.Nif(nif).forward(uv)
    B = nif.B.astype(np.float64)
    s = np.sin(2 * math.pi * (B[2, 0] * uv[:, 0] + B[2, 1] * uv[:, 1]))
    c = np.cos(2 * math.pi * (B[4, 0] * uv[:, 0] + B[4, 1] * uv[:, 1]))
    assert np.allclose(z[:, 1], s, atol=1e-12) and np.allclose(z[:, 0], c, atol=1e-12)
    assert np.allclose(z[:, 2], 0, atol=0)
    assert np.allclose(rgb[:, 1], np.exp(s), rtol=1e-12)


def _fd_check(nif, uv, target, delta, idx, h=1e-6):
    o = O.Nif(nif)
    loss, g = o.loss_grad(uv, target, delta)
    w0 = o.get_trainable()
    for i in idx:
        wp, wm = w0.copy(), w0.copy()
        wp[i] += h
        wm[i] -= h
        o.set_trainable(wp)
        lp, _ = o.loss_grad(uv, target, delta)
        o.set_trainable(wm)
        lm, _ = o.loss_grad(uv, target, delta)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1e-3 * np.abs(g).max()) + 1e-11, (i, fd, g[i])
    o.set_trainable(w0)
    return g


@pytest.mark.parametrize("delta", [10.0, 1e-3])
def test_gradient_matches_central_differences(delta):
    """Quadratic regime (delta large) and linear regime (delta small, targets
    far from the outputs) of the Huber loss."""
    nif = I.nif_init(n_freq=5, hidden=12, n_hidden_layers=3, colour="yuv", seed=2)
    rng = np.random.default_rng(2)
    for b in nif.b:
        b[:] = rng.normal(0, 0.1, b.shape)
    uv = rng.uniform(0, 1, (7, 2))
    target = rng.normal(0, 2, (7, 3))
    n = O.Nif(nif).n_trainable
    idx = list(range(0, n, max(1, n // 120))) + [n - 1, n - 2, n - 3]
    g = _fd_check(nif, uv, target, delta, idx)
    assert np.abs(g).max() > 0


def test_gradient_layout_matches_parameter_layout():
    """The gradient of the output bias for sample targets below the output
    (quadratic Huber) is the mean residual M^T (z - t) / 3."""
    nif = I.nif_init(n_freq=3, hidden=4, n_hidden_layers=1, colour="yuv")
    o = O.Nif(nif)
    uv = np.array([[0.2, 0.4], [0.6, 0.1]])
    rgb, z = o.forward(uv)
    t = z - 0.5
    loss, g = o.loss_grad(uv, t, delta=10.0)
    assert abs(loss - 0.5 * 0.25) < 1e-14
    db = g[-3:]
    want = nif.M.astype(np.float64).T @ np.full(3, 0.5) / 3.0
    assert np.allclose(db, want, atol=1e-15)


def test_adam_first_and_second_step_closed_form():
    """At t = 1 the bias-corrected moments are g and g^2, so the update is
    -lr g / (|g| + eps); at t = 2 with the same g it is the same again."""
    g = np.array([1e-2, -3.0, 5e-9, 0.0])
    w = np.zeros(4)
    m = np.zeros(4)
    v = np.zeros(4)
    O.adam_step(w, g.copy(), m, v, 1, lr=1e-3, eps=1e-7)
    want1 = -1e-3 * g / (np.abs(g) + 1e-7)
    assert np.allclose(w, want1, rtol=1e-14, atol=0)
    O.adam_step(w, g.copy(), m, v, 2, lr=1e-3, eps=1e-7)
    assert np.allclose(w, 2 * want1, rtol=1e-12, atol=1e-20)


def test_sky_bilinear_pixel_centres_wrap_and_clamp():
    rng = np.random.default_rng(0)
    sky = rng.uniform(0, 10, (6, 8, 3)).astype(np.float32)
    H, W = sky.shape[:2]
    # pixel centres reproduce the pixel values
    jj, ii = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
    uv = np.stack([(ii.ravel() + 0.5) / W, (jj.ravel() + 0.5) / H], 1)
    out = O.sky_bilinear(sky, uv)
    assert np.array_equal(out, sky.reshape(-1, 3).astype(np.float64))
    # u = 0 lies half way between the last and first column (wrap)
    out = O.sky_bilinear(sky, [[0.0, 2.5 / H]])
    assert np.allclose(out[0], 0.5 * (sky[2, 0] + sky[2, W - 1]))
    # v = 0 clamps to the top row
    out = O.sky_bilinear(sky, [[3.5 / W, 0.0]])
    assert np.allclose(out[0], sky[0, 3])
    # midpoint of four centres is their average
    out = O.sky_bilinear(sky, [[2.0 / W, 3.0 / H]])
    assert np.allclose(out[0], 0.25 * (sky[2, 1] + sky[2, 2] + sky[3, 1] + sky[3, 2]))


def test_procedural_sky_pixel_values():
    """Generator check at analytic pixel centres: zenith colour, ground, sun."""
    sky = I.procedural_sky(256, 128)
    assert np.all(sky[100, :, :] < 3.0)   # ground (v > 0.5), no lobes below the horizon
    assert sky.max() > 9e3                # sun disk present
    assert np.all(np.isfinite(sky)) and sky.min() > 0


def test_training_reduces_loss():
    """A short oracle training run on a small sky lowers the Huber loss."""
    nif = I.nif_init(n_freq=8, hidden=16, n_hidden_layers=2, colour="yuv")
    sky = I.procedural_sky(64, 32)
    o = O.Nif(nif)
    losses = o.train(sky, seed=0, steps=400, batch=128, lr=1e-2)
    assert losses[-20:].mean() < 0.75 * losses[:5].mean()


def test_ycocg_head_inverts_the_forward_transform():
    """The YCoCg head matrix maps (Y, Co, Cg) = (R/4 + G/2 + B/4, R/2 - B/2,
    -R/4 + G/2 - B/4) back to RGB exactly."""
    rgb = np.random.default_rng(3).uniform(-2, 2, (100, 3))
    R, G, B = rgb.T
    ycocg = np.stack([R / 4 + G / 2 + B / 4, R / 2 - B / 2, -R / 4 + G / 2 - B / 4], 1)
    back = ycocg @ I.YCOCG_TO_RGB.astype(np.float64).T
    assert np.allclose(back, rgb, atol=1e-12)
    assert np.array_equal(I.nif_init(colour="ycocg").M, I.YCOCG_TO_RGB)


# ---------------------------------------------------------------------------
# The paper's network shape: the Fourier features concatenated with the output
# of the last odd hidden layer before the middle (Section 3.2), whose width is
# reduced by 2F to keep the next layer's input at H.


def test_paper_network_has_97_kib_of_fp16_weights():
    """F = 20 (a 40-wide encoding), H = 128, four hidden ReLU layers and the
    head, the features joined to the output of hidden layer 2 (0-based odd
    layer 1, the last odd one before the middle): 50,011 parameters = 97.7 KiB
    in FP16, the size the paper quotes for its H128 network."""
    assert I.paper_skip_layer(4) == 2 and I.paper_skip_layer(5) == 2 and I.paper_skip_layer(8) == 4
    assert I.paper_skip_layer(2) == 0
    nif = I.nif_init(n_freq=20, hidden=128, n_hidden_layers=4, skip_after=I.paper_skip_layer(4))
    assert [W.shape for W in nif.W] == [(128, 40), (88, 128), (128, 128), (128, 128), (3, 128)]
    n = O.Nif(nif).n_trainable
    assert n == 50011 and 97.0 <= 2 * n / 1024 < 98.0


def test_skip_network_with_a_silent_skip_layer_is_the_shorter_plain_network():
    """If hidden layer s outputs nothing (zero weights and biases), layer
    s + 1 sees [0, features], so the network equals a plain network that
    starts at layer s + 1 with the feature columns of its weights."""
    F, H, L, s = 6, 32, 4, 2
    nif = I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L, skip_after=s, colour="yuv", seed=4)
    rng = np.random.default_rng(4)
    for b in nif.b:
        b[:] = rng.normal(0, 0.1, b.shape)
    nif.W[s - 1][:] = 0
    nif.b[s - 1][:] = 0
    short = I.NIF(nif.B.copy(), [nif.W[s][:, H - 2 * F:].copy()] + [W.copy() for W in nif.W[s + 1:]],
                  [b.copy() for b in nif.b[s:]], nif.M.copy())
    uv = rng.uniform(0, 1, (40, 2))
    a, _ = O.Nif(nif).forward(uv)
    b, _ = O.Nif(short).forward(uv)
    assert np.allclose(a, b, rtol=1e-13, atol=0)


def test_skip_network_passes_a_feature_around_the_skip_layer():
    """relu(x) - relu(-x) = x through the concatenated features only: the
    layers before the join are zero, layer s + 1 picks feature i from the
    appended block, the layers after pass it on, and the head returns it."""
    F, H, L, s = 4, 16, 3, 1
    nif = _zero_like(I.nif_init(n_freq=F, hidden=H, n_hidden_layers=L, skip_after=s))
    i = 3                                   # sin of frequency 3
    col = (H - 2 * F) + i                   # its column in layer s + 1's input
    nif.W[s][0, col], nif.W[s][1, col] = 1.0, -1.0
    nif.W[s + 1][0, 0], nif.W[s + 1][1, 1] = 1.0, 1.0
    nif.W[L][0, 0], nif.W[L][0, 1] = 1.0, -1.0
    uv = np.random.default_rng(5).uniform(0, 1, (30, 2)).astype(np.float32).astype(np.float64)
    _, z = O.Nif(nif).forward(uv)
    B = nif.B.astype(np.float64)
    want = np.sin(2 * math.pi * (B[i, 0] * uv[:, 0] + B[i, 1] * uv[:, 1]))
    assert np.allclose(z[:, 0], want, atol=1e-12)


@pytest.mark.parametrize("L,s", [(3, 1), (4, 2), (5, 3)])
def test_skip_network_gradient_matches_central_differences(L, s):
    nif = I.nif_init(n_freq=3, hidden=14, n_hidden_layers=L, skip_after=s, colour="yuv", seed=L)
    rng = np.random.default_rng(L)
    for b in nif.b:
        b[:] = rng.normal(0, 0.1, b.shape)
    uv = rng.uniform(0, 1, (6, 2))
    target = rng.normal(0, 2, (6, 3))
    n = O.Nif(nif).n_trainable
    idx = list(range(0, n, max(1, n // 150))) + [n - 1, n - 4]
    g = _fd_check(nif, uv, target, 10.0, idx)
    assert np.abs(g).max() > 0
