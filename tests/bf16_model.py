"""Rounding model of the tensor-core (BF16) training GEMMs, for the parity
tests: every GEMM operand is rounded to BF16 (round to nearest even) where
the kernels round it, sums run in FP64 (standing in for FP32 accumulation;
the difference is accumulation-order noise), everything else is FP64.

  forward   x[l+1] = relu(bf16(x[l]) bf16(W_l)^T + b_l)
  head      y = x[L] W_L^T + b_L in full precision, loss and dL/dy
  backward  G[L-1] = (dy W_L) * [x[L] > 0]
            G[l-1] = (bf16(G[l]) bf16(W_l)) * [bf16(x[l]) > 0]
  weights   dW_l = bf16(G[l])^T bf16(x[l]),  db_l = sum of bf16(G[l]) rows

With rounding switched off (`rounding=False`) the model is plain FP64
backpropagation, which the CPU tests check against the oracle's gradient
(Section 3.2.1 for the NIF loss, relative L2 for the radiance cache)."""
import numpy as np


def bf16(x):
    """FP32 -> nearest BF16 (ties to even), returned as FP32."""
    u = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    return ((u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000).astype(np.uint32).view(np.float32)


def _r(x, rounding):
    return bf16(np.asarray(x, np.float32)).astype(np.float64) if rounding else np.asarray(x, np.float64)


def nif_features(B, uv, fp32=True):
    """Layer-0 input of the NIF: [sin 2 pi (B uv), cos 2 pi (B uv)], the
    phase reduced to [-1/2, 1/2] from its FP64 value (the kernels carry B uv
    as an exact float pair, so their phase is as accurate).  fp32: features
    rounded to FP32 as the kernels store them."""
    uv = np.asarray(uv, np.float32)
    B = np.asarray(B, np.float64)
    t = (B[:, 0][None] * uv[:, :1].astype(np.float64) + B[:, 1][None] * uv[:, 1:].astype(np.float64))
    r = t - np.rint(t)
    f = np.concatenate([np.sin(2 * np.pi * r), np.cos(2 * np.pi * r)], 1)
    return f.astype(np.float32) if fp32 else f


def cache_features(cache, q, fp32=True):
    """Layer-0 input of the radiance cache: per axis sin / cos (pi 2^k p) of
    the box-normalised position, then wo and n (FP32 when fp32, else FP64)."""
    q = np.asarray(q, np.float64)
    lo, hi = cache.lo.astype(np.float64), cache.hi.astype(np.float64)
    p = (q[:, :3] - lo) / (hi - lo)
    feats = []
    for a in range(3):
        ang = np.pi * p[:, a:a + 1] * (2.0 ** np.arange(cache.n_freq))[None]
        feats += [np.sin(ang), np.cos(ang)]
    f = np.concatenate(feats + [q[:, 3:9]], 1)
    return f.astype(np.float32) if fp32 else f


def mlp_loss_grad(X0, Ws, bs, target, loss="huber", M=None, delta=1e-3, mask=None, rounding=True):
    """Loss (mean over n x 3) and the flat gradient (per layer W then b).
    loss "huber": Huber(delta) of M y against the target; "rel_l2": (y - t)^2
    / (y^2 + 0.01) with the denominator held constant, rows with mask == 0
    contributing nothing."""
    L = len(Ws) - 1
    n = X0.shape[0]
    xs = [np.asarray(X0, np.float64)]
    for l in range(L):
        a = _r(xs[l], rounding) @ _r(Ws[l], rounding).T + np.asarray(bs[l], np.float64)
        xs.append(np.maximum(a, 0.0))
    WL, bL = np.asarray(Ws[L], np.float64), np.asarray(bs[L], np.float64)
    y = xs[L] @ WL.T + bL
    t = np.asarray(target, np.float64)
    if loss == "huber":
        Mm = np.asarray(M, np.float64)
        z = y @ Mm.T
        r = z - t
        a = np.abs(r)
        lv = np.where(a <= delta, 0.5 * r * r, delta * (a - 0.5 * delta))
        dz = np.where(a <= delta, r, np.copysign(delta, r)) / (3.0 * n)
        dy = dz @ Mm
    else:
        r = y - t
        den = y * y + 0.01
        keep = np.ones(n, bool) if mask is None else np.asarray(mask) != 0
        lv = np.where(keep[:, None], r * r / den, 0.0)
        dy = np.where(keep[:, None], 2.0 * r / den, 0.0) / (3.0 * n)
    total = float(lv.sum() / (3.0 * n))
    grads = [None] * (L + 1)
    grads[L] = (dy.T @ xs[L], dy.sum(0))
    G = (dy @ WL) * (xs[L] > 0)
    for l in range(L - 1, -1, -1):
        Gb = _r(G, rounding)
        grads[l] = (Gb.T @ _r(xs[l], rounding), Gb.sum(0))
        if l > 0:
            G = (Gb @ _r(Ws[l], rounding)) * (_r(xs[l], rounding) > 0)
    flat = np.concatenate([np.concatenate([gw.ravel(), gb.ravel()]) for gw, gb in grads])
    return total, flat
