"""Shared helpers of the GPU parity tests (per-path comparison with the
FP64 oracle under the divergence reading)."""
import numpy as np
import torch

from oracle import oracle as O


def rel_rmse(img, ref):
    img = np.asarray(img, np.float64)
    ref = np.asarray(ref, np.float64)
    return float(np.sqrt(((img - ref) ** 2).sum() / (ref ** 2).sum()))


def subset_pixels(W, H):
    """Deterministic pixel subset (x + 7 y) mod 16 == 0."""
    y, x = np.divmod(np.arange(W * H), W)
    return np.where((x + 7 * y) % 16 == 0)[0].astype(np.int64)


def compare_render(pt, ctx, sc, cfg, nif=None, pixels=None, max_div=1e-3, tol=1e-3, max_div_v1=1e-4,
                   max_div_v2=1e-3, gpu_scene=None, oracle_scene=None, precision="fp32"):
    """Per-path parity with the oracle (same Philox streams).  A path is
    divergent when its hit-ID sequence differs from the oracle's.  Asserted:
    divergence at the primary hit <= max_div_v1, by vertex 2 <= max_div_v2,
    overall <= max_div, relative RMSE over matched paths <= tol."""
    s = gpu_scene if gpu_scene is not None else pt.Scene(ctx, sc)
    g = pt.Nif(ctx, nif) if nif is not None else None
    pix_t = None if pixels is None else torch.from_numpy(pixels).cuda()
    img, slots, ids = pt.render_pixels(ctx, s, g, cfg, pix_t, precision=precision, want_slots=True, want_ids=True)
    ctx.check()
    osc = oracle_scene if oracle_scene is not None else O.Scene(sc)
    r = O.render(osc, cfg, O.Nif(nif) if nif is not None else None, pixels=pixels, want_slots=True, want_ids=True)
    gslots = slots.cpu().numpy().transpose(1, 0, 2)
    gids = ids.cpu().numpy().transpose(1, 0, 2)
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
