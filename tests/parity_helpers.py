"""Shared helpers of the GPU parity tests (per-path comparison with the
FP64 oracle under the divergence reading)."""
import numpy as np
import torch

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I


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


def specular_vertices(sc, ids):
    """Number of metal or dielectric hits on each path (ids [n, D], -1 miss, -2 unused)."""
    prim_mat = np.concatenate([sc.sphere_mat, sc.quad_mat, sc.tri_mat])
    spec = np.isin(sc.mat_type[prim_mat], [I.METAL, I.DIELECTRIC])
    hit = ids >= 0
    return (hit & spec[np.where(hit, ids, 0)]).sum(1)


def conditioning_table(sc, ids_ref, L_ref, runs, max_bin=4):
    """Per specular-vertex count k of the reference path (k >= max_bin pooled):
    for each named run (L, ids), the fraction of divergent paths and the
    relative RMSE over matched paths."""
    ns = np.minimum(specular_vertices(sc, ids_ref), max_bin)
    rows = []
    for k in range(max_bin + 1):
        m = ns == k
        row = dict(k=k, n=int(m.sum()))
        for name, (L, ids) in runs.items():
            same = np.all(ids == ids_ref, axis=1)
            mm = m & same
            row[name + "_div"] = float(1 - same[m].mean()) if m.any() else 0.0
            row[name + "_matched"] = rel_rmse(L[mm], L_ref[mm]) if mm.any() else 0.0
        rows.append(row)
    return rows


def perturbed_camera(cam):
    """The camera moved by one float32 ulp along z (eye z -> the next float32
    towards +inf): the smallest change of the FP32 inputs, used to measure how
    strongly the FP64 paths themselves react to one rounding."""
    c = I.Camera.make(cam.eye.copy(), cam.target.copy(), cam.up.copy(), cam.fov_deg)
    c.eye[2] = np.nextafter(c.eye[2], np.float32(np.inf))
    return c


def assert_within_floor(rows, min_n=200, factor=3.0):
    """Each bin of a conditioning table with at least min_n paths: the GPU's
    divergent fraction within factor x the FP64 floor plus three binomial
    standard deviations, and its matched-path relative RMSE within factor x
    the floor's plus 1e-4."""
    for r in rows:
        if r["n"] < min_n:
            continue
        sd = np.sqrt(max(r["floor_div"], 1.0 / r["n"]) / r["n"])
        assert r["gpu_div"] <= factor * r["floor_div"] + 3 * sd, r
        assert r["gpu_matched"] <= factor * r["floor_matched"] + 1e-4, r
