"""ctypes binding of the FP64 CPU oracle.

TEST INFRASTRUCTURE ONLY: imported by tests/, ``__graft_entry__.smoke()`` and
the CPU-baseline leg of ``bench.py``.  The product path never imports this.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

from . import build as _build

_lib = None

P = C.c_void_p
I64 = C.c_int64
U32 = C.c_uint32


def _ptr(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        L.or_philox4x32_10.argtypes = [P, P, P]
        L.or_philox_batch.argtypes = [U32, U32, I64, P, P]
        L.or_scene_create.argtypes = [I64, P, P, I64, P, P, P, I64, P, I64, P, P, I64, P, P, C.c_int]
        L.or_scene_create.restype = P
        L.or_scene_destroy.argtypes = [P]
        L.or_scene_bvh_nodes.argtypes = [P]
        L.or_scene_bvh_nodes.restype = I64
        L.or_scene_bounds.argtypes = [P, P, P]
        L.or_closest_hit.argtypes = [P, I64, P, P, C.c_int, P, P]
        L.or_nif_create.argtypes = [C.c_int, C.c_int, C.c_int, P]
        L.or_nif_create.restype = P
        L.or_nif_create_skip.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, P]
        L.or_nif_create_skip.restype = P
        L.or_nif_destroy.argtypes = [P]
        L.or_nif_n_trainable.argtypes = [P]
        L.or_nif_n_trainable.restype = I64
        L.or_nif_export.argtypes = [P, P]
        L.or_nif_forward.argtypes = [P, I64, P, P, P]
        L.or_nif_loss_grad.argtypes = [P, I64, P, P, C.c_double, P]
        L.or_nif_loss_grad.restype = C.c_double
        L.or_adam_step.argtypes = [I64, P, P, P, P, I64, C.c_double, C.c_double, C.c_double, C.c_double]
        L.or_nif_get_trainable.argtypes = [P, P]
        L.or_nif_set_trainable.argtypes = [P, P]
        L.or_sky_bilinear.argtypes = [P, C.c_int, C.c_int, I64, P, P]
        L.or_train_uv.argtypes = [U32, U32, I64, P]
        L.or_nif_train.argtypes = [P, P, C.c_int, C.c_int, U32, I64, I64, C.c_double, C.c_double,
                                   C.c_double, C.c_double, C.c_double, P]
        L.or_primary_rays.argtypes = [P, C.c_int, C.c_int, U32, I64, P, P, P]
        L.or_dir_to_uv.argtypes = [I64, P, P]
        L.or_sample_bsdf.argtypes = [P, C.c_int, P, P, C.c_double, C.c_double, C.c_double, P, P]
        L.or_sample_bsdf.restype = C.c_int
        L.or_sample_bsdf_batch.argtypes = [P, C.c_int, P, P, I64, P, P, P, P]
        L.or_render.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_int, C.c_int, U32, C.c_int, C.c_int,
                                I64, P, P, P, P, C.c_int]
        _lib = L
    return _lib


# ----------------------------------------------------------------------------
def philox(ctr: Sequence[int], key: Sequence[int]) -> np.ndarray:
    c = np.asarray(ctr, np.uint32)
    k = np.asarray(key, np.uint32)
    out = np.zeros(4, np.uint32)
    lib().or_philox4x32_10(_ptr(c), _ptr(k), _ptr(out))
    return out


def philox_batch(seed: int, tag: int, ctr: np.ndarray) -> np.ndarray:
    ctr = np.ascontiguousarray(ctr, np.uint32).reshape(-1, 4)
    out = np.zeros_like(ctr)
    lib().or_philox_batch(seed, tag, len(ctr), _ptr(ctr), _ptr(out))
    return out


def camera_array(cam) -> np.ndarray:
    return np.concatenate([cam.eye, cam.target, cam.up, [cam.fov_deg]]).astype(np.float32)


class Scene:
    """Oracle-side copy of a scene (FP64), with the oracle's own BVH."""

    def __init__(self, scene, use_bvh: bool = True):
        scene.validate()
        self.src = scene
        self._keep = [scene.sphere, scene.sphere_mat, scene.quad, scene.quad_axis, scene.quad_mat,
                      scene.vert, scene.tri, scene.tri_mat, scene.mat_type, scene.mat]
        self.h = lib().or_scene_create(
            len(scene.sphere), _ptr(scene.sphere), _ptr(scene.sphere_mat),
            len(scene.quad), _ptr(scene.quad), _ptr(scene.quad_axis), _ptr(scene.quad_mat),
            len(scene.vert), _ptr(scene.vert), len(scene.tri), _ptr(scene.tri), _ptr(scene.tri_mat),
            len(scene.mat), _ptr(scene.mat_type), _ptr(scene.mat), int(use_bvh))

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_scene_destroy(self.h)
            self.h = None

    def bounds(self):
        lo = np.zeros(3)
        hi = np.zeros(3)
        lib().or_scene_bounds(self.h, _ptr(lo), _ptr(hi))
        return lo, hi

    def closest_hit(self, org: np.ndarray, dir: np.ndarray, brute: bool = False):
        org = np.ascontiguousarray(org, np.float64).reshape(-1, 3)
        dir = np.ascontiguousarray(dir, np.float64).reshape(-1, 3)
        t = np.zeros(len(org))
        ids = np.zeros(len(org), np.int64)
        lib().or_closest_hit(self.h, len(org), _ptr(org), _ptr(dir), int(brute), _ptr(t), _ptr(ids))
        return t, ids


def nif_flat(nif) -> np.ndarray:
    parts = [nif.B.ravel()]
    for W, b in zip(nif.W, nif.b):
        parts += [W.ravel(), b.ravel()]
    parts.append(nif.M.ravel())
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


class Nif:
    def __init__(self, nif):
        self.src = nif
        self.flat = nif_flat(nif)
        self.h = lib().or_nif_create_skip(nif.n_freq, nif.hidden, nif.n_hidden_layers, int(nif.skip_after),
                                          _ptr(self.flat))
        if not self.h:
            raise ValueError("unsupported NIF shape")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_nif_destroy(self.h)
            self.h = None

    @property
    def n_trainable(self) -> int:
        return int(lib().or_nif_n_trainable(self.h))

    def forward(self, uv: np.ndarray):
        uv = np.ascontiguousarray(uv, np.float64).reshape(-1, 2)
        rgb = np.zeros((len(uv), 3))
        z = np.zeros((len(uv), 3))
        lib().or_nif_forward(self.h, len(uv), _ptr(uv), _ptr(rgb), _ptr(z))
        return rgb, z

    def loss_grad(self, uv: np.ndarray, target: np.ndarray, delta: float = 1e-3):
        uv = np.ascontiguousarray(uv, np.float64).reshape(-1, 2)
        target = np.ascontiguousarray(target, np.float64).reshape(-1, 3)
        g = np.zeros(self.n_trainable)
        loss = lib().or_nif_loss_grad(self.h, len(uv), _ptr(uv), _ptr(target), float(delta), _ptr(g))
        return float(loss), g

    def get_trainable(self) -> np.ndarray:
        w = np.zeros(self.n_trainable)
        lib().or_nif_get_trainable(self.h, _ptr(w))
        return w

    def set_trainable(self, w: np.ndarray) -> None:
        w = np.ascontiguousarray(w, np.float64)
        assert w.size == self.n_trainable
        lib().or_nif_set_trainable(self.h, _ptr(w))

    def train(self, sky: np.ndarray, seed: int, steps: int, batch: int, lr=1e-3, beta1=0.9, beta2=0.999,
              eps=1e-7, delta=1e-3) -> np.ndarray:
        sky = np.ascontiguousarray(sky, np.float32)
        losses = np.zeros(steps)
        lib().or_nif_train(self.h, _ptr(sky), sky.shape[1], sky.shape[0], seed, steps, batch, lr, beta1, beta2,
                           eps, delta, _ptr(losses))
        return losses


def adam_step(w, g, m, v, t, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-7):
    for a in (w, g, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().or_adam_step(len(w), _ptr(w), _ptr(g), _ptr(m), _ptr(v), int(t), lr, beta1, beta2, eps)


def sky_bilinear(sky: np.ndarray, uv: np.ndarray) -> np.ndarray:
    sky = np.ascontiguousarray(sky, np.float32)
    uv = np.ascontiguousarray(uv, np.float64).reshape(-1, 2)
    out = np.zeros((len(uv), 3))
    lib().or_sky_bilinear(_ptr(sky), sky.shape[1], sky.shape[0], len(uv), _ptr(uv), _ptr(out))
    return out


def train_uv(seed: int, step: int, n: int) -> np.ndarray:
    uv = np.zeros((n, 2))
    lib().or_train_uv(seed, step, n, _ptr(uv))
    return uv


def primary_rays(cam, W: int, H: int, seed: int, slots: np.ndarray):
    slots = np.ascontiguousarray(slots, np.int64)
    ca = camera_array(cam)
    org = np.zeros((len(slots), 3))
    dir = np.zeros((len(slots), 3))
    lib().or_primary_rays(_ptr(ca), W, H, seed, len(slots), _ptr(slots), _ptr(org), _ptr(dir))
    return org, dir


def dir_to_uv(dirs: np.ndarray) -> np.ndarray:
    dirs = np.ascontiguousarray(dirs, np.float64).reshape(-1, 3)
    uv = np.zeros((len(dirs), 2))
    lib().or_dir_to_uv(len(dirs), _ptr(dirs), _ptr(uv))
    return uv


def render(oscene: Scene, cfg, nif: Optional[Nif] = None, pixels: Optional[np.ndarray] = None,
           want_slots: bool = False, want_ids: bool = False, n_threads: Optional[int] = None):
    """Render with the oracle.  Returns dict(image [n_pix, 3], slots, ids)."""
    sc = oscene.src
    cam = camera_array(sc.camera)
    env = None if sc.env_const is None else np.ascontiguousarray(sc.env_const, np.float32)
    if pixels is not None:
        pixels = np.ascontiguousarray(pixels, np.int64)
        n_pix = len(pixels)
    else:
        n_pix = cfg.width * cfg.height
    out = np.zeros((n_pix, 3))
    slots = np.zeros((n_pix, cfg.spp, 3)) if want_slots else None
    ids = np.zeros((n_pix, cfg.spp, cfg.max_depth), np.int64) if want_ids else None
    if n_threads is None:
        n_threads = os.cpu_count() or 1
    lib().or_render(oscene.h, nif.h if nif is not None else None, _ptr(env), _ptr(cam),
                    cfg.width, cfg.height, cfg.spp, cfg.max_depth, cfg.seed, int(cfg.rr), cfg.rr_start,
                    n_pix, _ptr(pixels), _ptr(out), _ptr(slots), _ptr(ids), int(n_threads))
    return dict(image=out, slots=slots, ids=ids)


def sample_bsdf(oscene: Scene, mat: int, d, ng, u1: float, u2: float, ul: float):
    d = np.ascontiguousarray(d, np.float64)
    ng = np.ascontiguousarray(ng, np.float64)
    wi = np.zeros(3)
    wt = np.zeros(3)
    ok = lib().or_sample_bsdf(oscene.h, mat, _ptr(d), _ptr(ng), u1, u2, ul, _ptr(wi), _ptr(wt))
    return bool(ok), wi, wt


def sample_bsdf_batch(oscene: Scene, mat: int, d, ng, u: np.ndarray):
    """sample_bsdf for every row (u1, u2, lobe) of u [n, 3]: (ok [n], wi [n, 3], weight [n, 3])."""
    d = np.ascontiguousarray(d, np.float64)
    ng = np.ascontiguousarray(ng, np.float64)
    u = np.ascontiguousarray(u, np.float64).reshape(-1, 3)
    n = len(u)
    wi = np.zeros((n, 3))
    wt = np.zeros((n, 3))
    ok = np.zeros(n, np.int32)
    lib().or_sample_bsdf_batch(oscene.h, mat, _ptr(d), _ptr(ng), n, _ptr(u), _ptr(wi), _ptr(wt), _ptr(ok))
    return ok.astype(bool), wi, wt


# ----------------------------------------------------------------------------
# radiance cache
def _cache_sigs(L):
    if getattr(L, "_cache_sigs", False):
        return
    L.or_cache_create.argtypes = [C.c_int, C.c_int, C.c_int, P, P]
    L.or_cache_create.restype = P
    L.or_cache_destroy.argtypes = [P]
    L.or_cache_n_params.argtypes = [P]
    L.or_cache_n_params.restype = I64
    L.or_cache_get_params.argtypes = [P, P]
    L.or_cache_set_params.argtypes = [P, P]
    L.or_cache_forward.argtypes = [P, I64, P, P]
    L.or_cache_loss_grad.argtypes = [P, I64, P, P, P, P, P]
    L.or_cache_loss_grad.restype = C.c_double
    L.or_trace_paths.argtypes = [P, P, P, P, C.c_int, C.c_int, C.c_int, U32, I64, P, P, P, C.c_int, C.c_int, P, P, P]
    L._cache_sigs = True


def cache_flat(cache) -> np.ndarray:
    parts = []
    for W, b in zip(cache.W, cache.b):
        parts += [W.ravel(), b.ravel()]
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


class Cache:
    """Oracle copy of a radiance cache (inputs.CacheNet)."""

    def __init__(self, cache):
        L = lib()
        _cache_sigs(L)
        self.src = cache
        self.flat = cache_flat(cache)
        self.bounds = np.ascontiguousarray(np.concatenate([cache.lo, cache.hi]).astype(np.float32))
        self.h = L.or_cache_create(cache.n_freq, cache.hidden, cache.n_hidden_layers, _ptr(self.flat), _ptr(self.bounds))
        if not self.h:
            raise ValueError("unsupported cache shape")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.or_cache_destroy(self.h)
            self.h = None

    @property
    def n_params(self) -> int:
        return int(lib().or_cache_n_params(self.h))

    def get_params(self) -> np.ndarray:
        w = np.zeros(self.n_params)
        lib().or_cache_get_params(self.h, _ptr(w))
        return w

    def set_params(self, w) -> None:
        w = np.ascontiguousarray(w, np.float64)
        lib().or_cache_set_params(self.h, _ptr(w))

    def forward(self, q: np.ndarray) -> np.ndarray:
        q = np.ascontiguousarray(q, np.float64).reshape(-1, 9)
        out = np.zeros((len(q), 3))
        lib().or_cache_forward(self.h, len(q), _ptr(q), _ptr(out))
        return out

    def loss_grad(self, q, target, denom=None, mask=None):
        q = np.ascontiguousarray(q, np.float64).reshape(-1, 9)
        target = np.ascontiguousarray(target, np.float64).reshape(-1, 3)
        denom = None if denom is None else np.ascontiguousarray(denom, np.float64).reshape(-1, 3)
        mask = None if mask is None else np.ascontiguousarray(mask, np.int32)
        g = np.zeros(self.n_params)
        loss = lib().or_cache_loss_grad(self.h, len(q), _ptr(q), _ptr(target), _ptr(denom), _ptr(mask), _ptr(g))
        return float(loss), g


def trace_paths(oscene: Scene, cam, W: int, H: int, depth: int, seed: int, pixels, samples, nif: Optional[Nif] = None,
                cache: Optional[Cache] = None, cache_vertex: int = 0, rec_vertex: int = 0, want_ids: bool = False):
    """Individual paths (pixel, sample): radiance [n,3], vertex records [n,16] (x, -d, n, tp, L before, valid)."""
    L = lib()
    _cache_sigs(L)
    sc = oscene.src
    pixels = np.ascontiguousarray(pixels, np.int64)
    samples = np.ascontiguousarray(samples, np.int64)
    n = len(pixels)
    env = None if sc.env_const is None else np.ascontiguousarray(sc.env_const, np.float32)
    ca = camera_array(cam)
    Lo = np.zeros((n, 3))
    rec = np.zeros((n, 16)) if rec_vertex else None
    ids = np.zeros((n, depth), np.int64) if want_ids else None
    L.or_trace_paths(oscene.h, nif.h if nif is not None else None, _ptr(env), _ptr(ca), W, H, depth, seed, n,
                     _ptr(pixels), _ptr(samples), cache.h if cache is not None else None, int(cache_vertex),
                     int(rec_vertex), _ptr(Lo), _ptr(rec), _ptr(ids))
    return Lo, rec, ids
