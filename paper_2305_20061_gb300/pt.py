"""Thin Python binding of the C ABI in include/pt.h.

Argument marshalling only: every step of the path runs in libpt.so's CUDA
kernels.  PyTorch supplies device memory (tensors' data pointers) and
streams.  Importing this module raises if the compiled library is missing;
there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np
import torch

from . import inputs as I

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpt.so")

PT_OK, PT_EINVAL, PT_ENOMEM, PT_ECUDA, PT_EDEVICE, PT_EUNSUPPORTED, PT_EIO = range(7)
PT_FP32, PT_BF16, PT_FP8E4M3 = 0, 1, 2
PRECISIONS = {"fp32": PT_FP32, "bf16": PT_BF16, "fp8": PT_FP8E4M3}
NODE_FORMATS = {"auto": 0, "packed": 1, "decoded": 2, "quant8": 3}
ERR_BITS = {0x1: "stack_overflow", 0x2: "queue_overflow", 0x4: "nonfinite", 0x8: "timeout", 0x10: "iter_cap",
            0x20: "bad_node", 0x80000000: "unreadable"}

P = C.c_void_p
I32 = C.c_int32
I64 = C.c_int64
U32 = C.c_uint32


class SceneDesc(C.Structure):
    _fields_ = [("n_spheres", I64), ("spheres", P), ("sphere_mat", P),
                ("n_quads", I64), ("quads", P), ("quad_axis", P), ("quad_mat", P),
                ("n_verts", I64), ("verts", P), ("n_tris", I64), ("tris", P), ("tri_mat", P),
                ("n_mats", I64), ("mat_type", P), ("mats", P),
                ("camera", C.c_float * 10), ("env_is_nif", I32), ("env_rgb", C.c_float * 3), ("node_format", I32)]


class SceneInfo(C.Structure):
    _fields_ = [("n_prims", I64), ("n_nodes", I64), ("node_bytes", I64), ("prim_bytes", I64),
                ("bvh_depth", I32), ("has_emission", I32), ("node_format", I32), ("reserved", I32),
                ("traversed_node_bytes", I64)]


class NifDesc(C.Structure):
    _fields_ = [("n_freq", I32), ("hidden", I32), ("n_hidden_layers", I32), ("params", P), ("skip_after", I32)]


class RenderCfg(C.Structure):
    _fields_ = [("width", I32), ("height", I32), ("spp", I32), ("max_depth", I32), ("seed", U32),
                ("rr", I32), ("rr_start", I32), ("precision", I32), ("chunk_slots", I64),
                ("first_sample", I32), ("schedule", I32), ("cache_vertex", I32)]


class TrainCfg(C.Structure):
    _fields_ = [("steps", I64), ("batch", I64), ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float),
                ("eps", C.c_float), ("huber_delta", C.c_float), ("seed", U32), ("precision", I32)]


class CacheDesc(C.Structure):
    _fields_ = [("n_freq", I32), ("hidden", I32), ("n_hidden_layers", I32), ("params", P),
                ("lo", C.c_float * 3), ("hi", C.c_float * 3)]


class CacheTrainCfg(C.Structure):
    _fields_ = [("width", I32), ("height", I32), ("n_train", I32), ("max_depth", I32), ("rec_vertex", I32),
                ("seed", U32), ("frame", U32), ("precision", I32), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("train_precision", I32)]


class CheckpointInfo(C.Structure):
    _fields_ = [("kind", I32), ("version", I32), ("dims", I32 * 4), ("lo", C.c_float * 3), ("hi", C.c_float * 3),
                ("n_params", I64), ("n_adam", I64), ("adam_t", I64)]


class PTError(RuntimeError):
    def __init__(self, status: int, msg: str, bits: int = 0):
        super().__init__(f"pt status {status}: {msg}")
        self.status = status
        self.bits = bits


_lib = None


def lib():
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2305_20061_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        sig = {
            "pt_create": ([P, C.c_int], I32),
            "pt_destroy": ([P], None),
            "pt_last_error": ([P], C.c_char_p),
            "pt_check": ([P, P, P], I32),
            "pt_create_scene": ([P, P, P], I32),
            "pt_destroy_scene": ([P], None),
            "pt_scene_get_info": ([P, P], I32),
            "pt_scene_download_bvh": ([P, P, P, P], I32),
            "pt_load_nif": ([P, P, P], I32),
            "pt_destroy_nif": ([P], None),
            "pt_nif_param_count": ([P], I64),
            "pt_nif_get_params": ([P, P, P], I32),
            "pt_nif_eval": ([P, P, I32, I64, P, P, P], I32),
            "pt_render": ([P, P, P, P, P, P, P], I32),
            "pt_device_error_bits": ([P], U32),
            "pt_microbench_ffma": ([I64, P, P, P], I32),
            "pt_microbench_l2_read": ([P, I64, I32, P, P, P], I32),
            "pt_render_pixels": ([P, P, P, P, I64, P, P, P, P, P], I32),
            "pt_last_render_counts": ([P, P, I32], I32),
            "pt_philox": ([P, U32, U32, I64, P, P, P], I32),
            "pt_primary_rays": ([P, P, P, I64, I64, P, P, P], I32),
            "pt_trace_rays": ([P, P, I64, P, P, P, P, P], I32),
            "pt_profile_enable": ([P, I32], I32),
            "pt_profile_read": ([P, P, P, I32], I32),
            "pt_render_noalloc": ([P, P, P, P, P, P], I32),
            "pt_last_render_work": ([P, P, I32], I32),
            "pt_last_render_schedule": ([P, P], I32),
            "pt_kernel_launches": ([P], I32),
            "pt_build_bvh_host": ([I64, P, P, P, I64, P, P, P], I32),
            "pt_quantize_bvh_host": ([I64, P, P], I32),
            "pt_nif_set_params": ([P, P, P, P], I32),
            "pt_nif_fp8_scales": ([P, P], I32),
            "pt_train_nif": ([P, P, P, I32, I32, P, P, P], I32),
            "pt_nif_loss_grad": ([P, P, I64, P, P, C.c_float, I32, P, P, P], I32),
            "pt_create_cache": ([P, P, P], I32),
            "pt_destroy_cache": ([P], None),
            "pt_cache_param_count": ([P], I64),
            "pt_cache_get_params": ([P, P, P], I32),
            "pt_cache_set_params": ([P, P, P, P], I32),
            "pt_cache_eval": ([P, P, I32, I64, P, P, P], I32),
            "pt_cache_loss_grad": ([P, P, I64, P, P, P, I32, P, P, P], I32),
            "pt_train_cache": ([P, P, P, P, P, P, P], I32),
            "pt_render_cached": ([P, P, P, P, I32, I32, P, I64, P, P, P, P, P, P], I32),
            "pt_save_nif": ([P, P, C.c_char_p, P], I32),
            "pt_load_nif_file": ([P, C.c_char_p, P], I32),
            "pt_save_cache": ([P, P, C.c_char_p, P], I32),
            "pt_load_cache_file": ([P, C.c_char_p, P], I32),
            "pt_checkpoint_read_info": ([C.c_char_p, P], I32),
            "pt_selftest_wait_timeout": ([P, C.c_double, P, P], I32),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
    return _lib


def _np_ptr(a: Optional[np.ndarray]):
    return None if a is None or a.size == 0 else a.ctypes.data_as(P)


def _dptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "device tensors must be contiguous CUDA tensors"
    return P(t.data_ptr())


def _stream(stream) -> P:
    if stream is None:
        stream = torch.cuda.current_stream()
    return P(stream.cuda_stream)


class Context:
    """A library context on one CUDA device (pt_create / pt_destroy)."""

    def __init__(self, device: int = 0):
        self.h = P()
        st = lib().pt_create(C.byref(self.h), int(device))
        if st != PT_OK:
            raise PTError(st, "pt_create failed")
        self.device = device

    def _raise(self, st: int):
        if st != PT_OK:
            raise PTError(st, lib().pt_last_error(self.h).decode())

    def check(self, stream=None) -> int:
        """Synchronise and read (and clear) the device error word."""
        bits = U32(0)
        st = lib().pt_check(self.h, _stream(stream), C.byref(bits))
        if st not in (PT_OK, PT_EDEVICE):
            self._raise(st)
        if st == PT_EDEVICE:
            names = [n for b, n in ERR_BITS.items() if bits.value & b]
            raise PTError(st, "device error bits " + ",".join(names), bits.value)
        return bits.value

    def selftest_wait_timeout(self, seconds: float = 0.05, stream=None) -> float:
        """pt_selftest_wait_timeout: a bounded device wait that nothing satisfies gives up after `seconds` and
        sets PT_ERR_TIMEOUT (read by the next check()); returns the time the device waited."""
        waited = C.c_double(0.0)
        self._raise(lib().pt_selftest_wait_timeout(self.h, float(seconds), C.byref(waited), _stream(stream)))
        return waited.value

    def close(self):
        if self.h:
            lib().pt_destroy(self.h)
            self.h = P()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """pt_create_scene from an inputs.Scene (host arrays, read during the call)."""

    def __init__(self, ctx: Context, scene: I.Scene, node_format: str = "auto"):
        scene.validate()
        self.ctx = ctx
        self.src = scene
        d = SceneDesc()
        d.n_spheres, d.spheres, d.sphere_mat = len(scene.sphere), _np_ptr(scene.sphere), _np_ptr(scene.sphere_mat)
        d.n_quads, d.quads, d.quad_axis, d.quad_mat = (len(scene.quad), _np_ptr(scene.quad),
                                                       _np_ptr(scene.quad_axis), _np_ptr(scene.quad_mat))
        d.n_verts, d.verts = len(scene.vert), _np_ptr(scene.vert)
        d.n_tris, d.tris, d.tri_mat = len(scene.tri), _np_ptr(scene.tri), _np_ptr(scene.tri_mat)
        d.n_mats, d.mat_type, d.mats = len(scene.mat), _np_ptr(scene.mat_type), _np_ptr(scene.mat)
        cam = np.concatenate([scene.camera.eye, scene.camera.target, scene.camera.up, [scene.camera.fov_deg]])
        for i in range(10):
            d.camera[i] = float(cam[i])
        d.env_is_nif = 0 if scene.env_const is not None else 1
        env = scene.env_const if scene.env_const is not None else np.zeros(3)
        for i in range(3):
            d.env_rgb[i] = float(env[i])
        d.node_format = NODE_FORMATS[node_format]
        self.h = P()
        ctx._raise(lib().pt_create_scene(ctx.h, C.byref(d), C.byref(self.h)))

    def info(self) -> dict:
        inf = SceneInfo()
        self.ctx._raise(lib().pt_scene_get_info(self.h, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in SceneInfo._fields_}

    def download_bvh(self):
        n = self.info()["n_nodes"]
        nodes = np.zeros((max(n, 1), 12), np.uint32)
        root = U32(0)
        self.ctx._raise(lib().pt_scene_download_bvh(self.ctx.h, self.h, _np_ptr(nodes), C.byref(root)))
        return nodes[:n], root.value

    def __del__(self):
        if getattr(self, "h", None):
            lib().pt_destroy_scene(self.h)
            self.h = None


def nif_flat(nif: I.NIF) -> np.ndarray:
    """Flat float32 parameter layout of include/pt.h (B, per layer W and b, M)."""
    parts = [nif.B.ravel()]
    for W, b in zip(nif.W, nif.b):
        parts += [W.ravel(), b.ravel()]
    parts.append(nif.M.ravel())
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


def nif_from_flat(F: int, H: int, L: int, flat: np.ndarray, skip_after: int = 0) -> I.NIF:
    """Inverse of nif_flat for a NIF of n_freq F, hidden width H, L hidden layers and skip layer skip_after."""
    p = 0
    B = flat[p:p + 2 * F].reshape(F, 2).copy()
    p += 2 * F
    Ws, bs = [], []
    for l in range(L + 1):
        i, o = (2 * F if l == 0 else H), (3 if l == L else (H - 2 * F if skip_after and l == skip_after - 1 else H))
        Ws.append(flat[p:p + i * o].reshape(o, i).copy())
        p += i * o
        bs.append(flat[p:p + o].copy())
        p += o
    return I.NIF(B, Ws, bs, flat[p:p + 9].reshape(3, 3).copy(), int(skip_after))


def checkpoint_info(path: str) -> dict:
    """pt_checkpoint_read_info: header of a verified checkpoint file (no device needed)."""
    inf = CheckpointInfo()
    st = lib().pt_checkpoint_read_info(os.fsencode(path), C.byref(inf))
    if st != PT_OK:
        raise PTError(st, f"checkpoint {path} unreadable")
    return {"kind": {1: "nif", 2: "cache"}.get(inf.kind, inf.kind), "version": inf.version, "dims": list(inf.dims),
            "lo": list(inf.lo), "hi": list(inf.hi), "n_params": inf.n_params, "n_adam": inf.n_adam,
            "adam_t": inf.adam_t}


class Nif:
    """pt_load_nif from an inputs.NIF (or Nif.load from a checkpoint file)."""

    def __init__(self, ctx: Context, nif: I.NIF):
        self.ctx = ctx
        self.src = nif
        flat = nif_flat(nif)
        d = NifDesc(nif.n_freq, nif.hidden, nif.n_hidden_layers, _np_ptr(flat), int(nif.skip_after))
        self.h = P()
        ctx._raise(lib().pt_load_nif(ctx.h, C.byref(d), C.byref(self.h)))

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Nif":
        """pt_load_nif_file: weights and training state from a checkpoint."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.h = P()
        ctx._raise(lib().pt_load_nif_file(ctx.h, os.fsencode(path), C.byref(self.h)))
        F, H, L, S = checkpoint_info(path)["dims"][:4]
        self.src = nif_from_flat(F, H, L, self.get_params(), S)
        return self

    def save(self, path: str, stream=None) -> None:
        """pt_save_nif: weights and (once training started) Adam state to a checkpoint file."""
        self.ctx._raise(lib().pt_save_nif(self.ctx.h, self.h, os.fsencode(path), _stream(stream)))

    @property
    def param_count(self) -> int:
        return int(lib().pt_nif_param_count(self.h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count, np.float32)
        self.ctx._raise(lib().pt_nif_get_params(self.ctx.h, self.h, _np_ptr(out)))
        return out

    def fp8_scales(self) -> np.ndarray:
        out = np.zeros(4, np.float32)
        self.ctx._raise(lib().pt_nif_fp8_scales(self.h, _np_ptr(out)))
        return out

    def set_params(self, flat: np.ndarray, stream=None) -> None:
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.param_count
        self.ctx._raise(lib().pt_nif_set_params(self.ctx.h, self.h, _np_ptr(flat), _stream(stream)))

    def train(self, sky: torch.Tensor, steps: int, batch: int = 1 << 16, lr: float = 1e-3, beta1: float = 0.9,
              beta2: float = 0.999, eps: float = 1e-7, delta: float = 1e-3, seed: int = 0, precision: str = "fp32",
              stream=None) -> torch.Tensor:
        """pt_train_nif on an HDR image [h, w, 3] (device tensor); returns per-step losses.  precision: the
        training GEMMs, "fp32" (CUDA cores) or "bf16" (tensor cores, BF16 operands, FP32 accumulation)."""
        sky = sky.contiguous()
        losses = torch.zeros(max(steps, 1), dtype=torch.float32, device=sky.device)
        cfg = TrainCfg(steps, batch, lr, beta1, beta2, eps, delta, seed, PRECISIONS[precision])
        self.ctx._raise(lib().pt_train_nif(self.ctx.h, self.h, _dptr(sky), sky.shape[1], sky.shape[0], C.byref(cfg),
                                           _dptr(losses), _stream(stream)))
        return losses[:steps]

    def loss_grad(self, uv: torch.Tensor, target: torch.Tensor, delta: float = 1e-3, precision: str = "fp32",
                  stream=None):
        """pt_nif_loss_grad: (loss as a device double tensor, gradient in the trainable flat layout)."""
        uv, target = uv.contiguous(), target.contiguous()
        n_tr = self.param_count - 2 * self.src.n_freq - 9
        grad = torch.empty(n_tr, dtype=torch.float32, device=uv.device)
        loss = torch.zeros(1, dtype=torch.float64, device=uv.device)
        self.ctx._raise(lib().pt_nif_loss_grad(self.ctx.h, self.h, uv.shape[0], _dptr(uv), _dptr(target), delta,
                                               PRECISIONS[precision], _dptr(grad), _dptr(loss), _stream(stream)))
        return loss, grad

    def eval(self, uv: torch.Tensor, precision: str = "fp32", stream=None) -> torch.Tensor:
        uv = uv.contiguous()
        rgb = torch.empty((uv.shape[0], 3), dtype=torch.float32, device=uv.device)
        self.ctx._raise(lib().pt_nif_eval(self.ctx.h, self.h, PRECISIONS[precision], uv.shape[0], _dptr(uv),
                                          _dptr(rgb), _stream(stream)))
        return rgb

    def __del__(self):
        if getattr(self, "h", None):
            lib().pt_destroy_nif(self.h)
            self.h = None


def cache_flat(cache: I.CacheNet) -> np.ndarray:
    """Flat float32 parameter layout of pt_cache_desc (per layer W then b)."""
    parts = []
    for W, b in zip(cache.W, cache.b):
        parts += [W.ravel(), b.ravel()]
    return np.ascontiguousarray(np.concatenate(parts).astype(np.float32))


class Cache:
    """pt_create_cache from an inputs.CacheNet (or Cache.load from a checkpoint file)."""

    def __init__(self, ctx: Context, cache: I.CacheNet):
        self.ctx = ctx
        self.src = cache
        flat = cache_flat(cache)
        d = CacheDesc(cache.n_freq, cache.hidden, cache.n_hidden_layers, _np_ptr(flat))
        for a in range(3):
            d.lo[a] = float(cache.lo[a])
            d.hi[a] = float(cache.hi[a])
        self.h = P()
        ctx._raise(lib().pt_create_cache(ctx.h, C.byref(d), C.byref(self.h)))

    @classmethod
    def load(cls, ctx: Context, path: str) -> "Cache":
        """pt_load_cache_file: weights, box and training state from a checkpoint (a per-frame snapshot)."""
        self = cls.__new__(cls)
        self.ctx = ctx
        self.h = P()
        ctx._raise(lib().pt_load_cache_file(ctx.h, os.fsencode(path), C.byref(self.h)))
        info = checkpoint_info(path)
        J, H, L = info["dims"][:3]
        flat = self.get_params()
        Ws, bs, p = [], [], 0
        for l in range(L + 1):
            i, o = (6 * J + 6 if l == 0 else H), (3 if l == L else H)
            Ws.append(flat[p:p + i * o].reshape(o, i).copy())
            p += i * o
            bs.append(flat[p:p + o].copy())
            p += o
        self.src = I.CacheNet(J, Ws, bs, np.array(info["lo"], np.float32), np.array(info["hi"], np.float32))
        return self

    def save(self, path: str, stream=None) -> None:
        """pt_save_cache: weights, box and (once training started) Adam state to a checkpoint file."""
        self.ctx._raise(lib().pt_save_cache(self.ctx.h, self.h, os.fsencode(path), _stream(stream)))

    @property
    def param_count(self) -> int:
        return int(lib().pt_cache_param_count(self.h))

    def get_params(self) -> np.ndarray:
        out = np.zeros(self.param_count, np.float32)
        self.ctx._raise(lib().pt_cache_get_params(self.ctx.h, self.h, _np_ptr(out)))
        return out

    def set_params(self, flat: np.ndarray, stream=None) -> None:
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.param_count
        self.ctx._raise(lib().pt_cache_set_params(self.ctx.h, self.h, _np_ptr(flat), _stream(stream)))

    def eval(self, q: torch.Tensor, precision: str = "fp32", stream=None) -> torch.Tensor:
        """pt_cache_eval: raw outputs [n, 3] for queries [n, 9] (x, wo, n)."""
        q = q.contiguous()
        out = torch.empty((q.shape[0], 3), dtype=torch.float32, device=q.device)
        self.ctx._raise(lib().pt_cache_eval(self.ctx.h, self.h, PRECISIONS[precision], q.shape[0], _dptr(q),
                                            _dptr(out), _stream(stream)))
        return out

    def loss_grad(self, q: torch.Tensor, target: torch.Tensor, mask: Optional[torch.Tensor] = None,
                  precision: str = "fp32", stream=None):
        """pt_cache_loss_grad: (loss as a device double tensor, flat gradient); precision of the GEMMs."""
        q, target = q.contiguous(), target.contiguous()
        grad = torch.empty(self.param_count, dtype=torch.float32, device=q.device)
        loss = torch.zeros(1, dtype=torch.float64, device=q.device)
        self.ctx._raise(lib().pt_cache_loss_grad(self.ctx.h, self.h, q.shape[0], _dptr(q), _dptr(target),
                                                 _dptr(None if mask is None else mask.contiguous()),
                                                 PRECISIONS[precision], _dptr(grad), _dptr(loss), _stream(stream)))
        return loss, grad

    def train_frame(self, scene: "Scene", nif: Optional["Nif"], width: int, height: int, frame: int,
                    n_train: int = 1 << 16, max_depth: int = 6, rec_vertex: int = 2, seed: int = 0,
                    precision: str = "fp32", lr: float = 1e-2, beta1: float = 0.9, beta2: float = 0.999,
                    eps: float = 1e-7, loss: Optional[torch.Tensor] = None, train_precision: str = "fp32",
                    stream=None) -> Optional[torch.Tensor]:
        """pt_train_cache: one online training step; loss (optional [1] float32 device tensor) receives the loss.
        precision: the NIF at the training paths' escapes; train_precision: the network's training GEMMs."""
        cfg = CacheTrainCfg(width, height, n_train, max_depth, rec_vertex, seed, frame, PRECISIONS[precision], lr,
                            beta1, beta2, eps, PRECISIONS[train_precision])
        self.ctx._raise(lib().pt_train_cache(self.ctx.h, scene.h, nif.h if nif is not None else None, self.h,
                                             C.byref(cfg), _dptr(loss), _stream(stream)))
        return loss

    def __del__(self):
        if getattr(self, "h", None):
            lib().pt_destroy_cache(self.h)
            self.h = None


# pt_schedule: automatic, one launch per vertex (wavefront), one launch per chunk (path per thread)
SCHEDULES = {"auto": 0, "wavefront": 1, "paths": 2}


def make_cfg(cfg: I.RenderCfg, precision: str = "fp32", chunk_slots: int = 0, first_sample: int = 0,
             schedule: str = "auto", cache_vertex: int = 0) -> RenderCfg:
    return RenderCfg(cfg.width, cfg.height, cfg.spp, cfg.max_depth, cfg.seed, int(cfg.rr), cfg.rr_start,
                     PRECISIONS[precision], int(chunk_slots), int(first_sample), SCHEDULES[schedule],
                     int(cache_vertex))


KINDS = ("trace", "nif", "reduce", "other", "cache", "shade")


def profile_enable(ctx: Context, enable: bool = True) -> None:
    ctx._raise(lib().pt_profile_enable(ctx.h, int(enable)))


def profile_read(ctx: Context) -> dict:
    """Device milliseconds and launch counts per kernel kind since the last read."""
    ms = np.zeros(len(KINDS))
    n = np.zeros(len(KINDS), np.int64)
    ctx._raise(lib().pt_profile_read(ctx.h, _np_ptr(ms), _np_ptr(n), len(KINDS)))
    return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(KINDS)}


def render(ctx: Context, scene: Scene, nif: Optional[Nif], cfg: I.RenderCfg, precision: str = "fp32",
           out: Optional[torch.Tensor] = None, chunk_slots: int = 0, first_sample: int = 0,
           stream=None, schedule: str = "auto", cache: Optional["Cache"] = None,
           cache_vertex: int = 0) -> torch.Tensor:
    """pt_render: returns the [H, W, 3] float32 image on the context's device
    (with a radiance cache, paths end in it at cache_vertex)."""
    if out is None:
        out = torch.empty((cfg.height, cfg.width, 3), dtype=torch.float32, device=f"cuda:{ctx.device}")
    c = make_cfg(cfg, precision, chunk_slots, first_sample, schedule, cache_vertex)
    ctx._raise(lib().pt_render(ctx.h, scene.h, nif.h if nif is not None else None,
                               cache.h if cache is not None else None, C.byref(c), _dptr(out), _stream(stream)))
    return out


def l2_read_rate_gbs(device: int, mib: int = 48, reps: int = 20, trials: int = 3) -> float:
    """L2 read bandwidth of the device in GB/s: pt_microbench_l2_read over a
    buffer of `mib` MiB (inside L2), timed with CUDA events on the current
    stream (best of `trials` after one warm-up launch)."""
    dev = f"cuda:{device}"
    buf = torch.zeros(mib << 18, dtype=torch.float32, device=dev)   # mib MiB
    sink = torch.zeros(1, dtype=torch.int32, device=dev)
    nbytes = C.c_double(0)
    s = torch.cuda.current_stream(device)
    best = 0.0
    for i in range(trials + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = lib().pt_microbench_l2_read(_dptr(buf), buf.numel() * 4, reps, _dptr(sink), C.byref(nbytes), _stream(s))
        e1.record(s)
        if st != PT_OK:
            raise PTError(st, "pt_microbench_l2_read failed")
        torch.cuda.synchronize(dev)
        if i:
            best = max(best, nbytes.value / (e0.elapsed_time(e1) * 1e-3) / 1e9)
    return best


def ffma_rate_tflops(device: int, iters: int = 1 << 16, reps: int = 3) -> float:
    """FP32 FMA rate of the device in TFLOP/s: pt_microbench_ffma timed with
    CUDA events on the current stream (best of reps, after one warm-up)."""
    dev = f"cuda:{device}"
    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    flop = C.c_double(0)
    s = torch.cuda.current_stream(device)
    best = 0.0
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        st = lib().pt_microbench_ffma(iters, _dptr(sink), C.byref(flop), _stream(s))
        e1.record(s)
        if st != PT_OK:
            raise PTError(st, "pt_microbench_ffma failed")
        torch.cuda.synchronize(dev)
        if i:
            best = max(best, flop.value / (e0.elapsed_time(e1) * 1e-3) / 1e12)
    return best


def device_error_bits(ctx: Context) -> int:
    """pt_device_error_bits: the context's device error word, not cleared."""
    return int(lib().pt_device_error_bits(ctx.h))


def render_pixels(ctx: Context, scene: Scene, nif: Optional[Nif], cfg: I.RenderCfg, pixels: Optional[torch.Tensor],
                  precision: str = "fp32", want_slots: bool = False, want_ids: bool = False, chunk_slots: int = 0,
                  stream=None, schedule: str = "auto"):
    """pt_render_pixels: (pixel_rgb [n,3], slot_rgb [spp,n,3] or None, hit_ids [spp,n,D] or None)."""
    dev = f"cuda:{ctx.device}"
    n = cfg.width * cfg.height if pixels is None else int(pixels.shape[0])
    pix = torch.empty((n, 3), dtype=torch.float32, device=dev)
    slots = torch.empty((cfg.spp, n, 3), dtype=torch.float32, device=dev) if want_slots else None
    ids = torch.empty((cfg.spp, n, cfg.max_depth), dtype=torch.int32, device=dev) if want_ids else None
    c = make_cfg(cfg, precision, chunk_slots, schedule=schedule)
    ctx._raise(lib().pt_render_pixels(ctx.h, scene.h, nif.h if nif is not None else None, C.byref(c), n,
                                      _dptr(pixels), _dptr(pix), _dptr(slots), _dptr(ids), _stream(stream)))
    return pix, slots, ids


def render_cached(ctx: Context, scene: Scene, nif: Optional[Nif], cfg: I.RenderCfg, pixels: Optional[torch.Tensor],
                  cache: Optional[Cache] = None, cache_vertex: int = 0, rec_vertex: int = 0, precision: str = "fp32",
                  want_slots: bool = False, want_ids: bool = False, chunk_slots: int = 0, first_sample: int = 0,
                  out: Optional[torch.Tensor] = None, stream=None, schedule: str = "auto"):
    """pt_render_cached: (pixel_rgb [n,3], slot_rgb [spp,n,3] or None, records [spp,n,16] or None,
    hit_ids [spp,n,D] or None).  out (optional): preallocated pixel_rgb."""
    dev = f"cuda:{ctx.device}"
    n = cfg.width * cfg.height if pixels is None else int(pixels.shape[0])
    pix = out if out is not None else torch.empty((n, 3), dtype=torch.float32, device=dev)
    slots = torch.empty((cfg.spp, n, 3), dtype=torch.float32, device=dev) if want_slots else None
    rec = torch.empty((cfg.spp, n, 16), dtype=torch.float32, device=dev) if rec_vertex else None
    ids = torch.empty((cfg.spp, n, cfg.max_depth), dtype=torch.int32, device=dev) if want_ids else None
    c = make_cfg(cfg, precision, chunk_slots, first_sample, schedule)
    ctx._raise(lib().pt_render_cached(ctx.h, scene.h, nif.h if nif is not None else None,
                                      cache.h if cache is not None else None, cache_vertex, rec_vertex, C.byref(c), n,
                                      _dptr(pixels), _dptr(pix), _dptr(slots), _dptr(rec), _dptr(ids),
                                      _stream(stream)))
    return pix, slots, rec, ids


def last_render_counts(ctx: Context, max_depth: int, with_cache: bool = False) -> np.ndarray:
    """Rays traced per vertex, then NIF evaluations (and cache queries with with_cache)."""
    out = np.zeros(max_depth + 1 + int(with_cache), np.int64)
    ctx._raise(lib().pt_last_render_counts(ctx.h, _np_ptr(out), len(out)))
    return out


def build_bvh_host(lo: np.ndarray, hi: np.ndarray):
    """pt_build_bvh_host: the scene builder's BVH from primitive boxes
    [n, 3] on the host.  Returns (nodes [n - 1, 12] uint32, root, depth)."""
    lo = np.ascontiguousarray(lo, np.float32)
    hi = np.ascontiguousarray(hi, np.float32)
    n = int(lo.shape[0])
    nodes = np.zeros((max(n - 1, 1), 12), np.uint32)
    n_nodes, root, depth = C.c_int64(0), C.c_uint32(0), C.c_int32(0)
    st = lib().pt_build_bvh_host(n, _np_ptr(lo), _np_ptr(hi), _np_ptr(nodes), nodes.shape[0], C.byref(n_nodes),
                                 C.byref(root), C.byref(depth))
    if st != PT_OK:
        raise PTError(st, "pt_build_bvh_host failed")
    return nodes[:n_nodes.value], int(root.value), int(depth.value)


def quantize_bvh_host(nodes: np.ndarray) -> np.ndarray:
    """pt_quantize_bvh_host: the 32-byte quantised form [n, 8] uint32 of packed nodes [n, 12]."""
    nodes = np.ascontiguousarray(nodes, np.uint32).reshape(-1, 12)
    out = np.zeros((max(len(nodes), 1), 8), np.uint32)
    st = lib().pt_quantize_bvh_host(len(nodes), _np_ptr(nodes), _np_ptr(out))
    if st != PT_OK:
        raise PTError(st, "pt_quantize_bvh_host failed")
    return out[:len(nodes)]


def kernel_launches() -> int:
    """Kernels the library has launched in this process (graph replays included)."""
    v = C.c_uint64(0)
    st = lib().pt_kernel_launches(C.byref(v))
    if st != PT_OK:
        raise PTError(st, "pt_kernel_launches failed")
    return int(v.value)


def last_render_schedule(ctx: Context) -> str:
    """"wavefront" or "paths": how the last render's last chunk was scheduled."""
    v = C.c_int32(0)
    ctx._raise(lib().pt_last_render_schedule(ctx.h, C.byref(v)))
    return {v_: k for k, v_ in SCHEDULES.items()}[v.value]


def last_render_work(ctx: Context) -> dict:
    """Traversal work of the last render: node fetches and primitive tests."""
    out = np.zeros(4, np.int64)
    ctx._raise(lib().pt_last_render_work(ctx.h, _np_ptr(out), 4))
    return dict(nodes=int(out[0]), sphere=int(out[1]), quad=int(out[2]), triangle=int(out[3]))


def philox(ctx: Context, seed: int, tag: int, ctr: torch.Tensor, stream=None) -> torch.Tensor:
    ctr = ctr.contiguous()
    out = torch.empty_like(ctr)
    ctx._raise(lib().pt_philox(ctx.h, seed, tag, ctr.shape[0], _dptr(ctr), _dptr(out), _stream(stream)))
    return out


def primary_rays(ctx: Context, scene: Scene, cfg: I.RenderCfg, first_slot: int, n: int, stream=None):
    dev = f"cuda:{ctx.device}"
    org = torch.empty((n, 3), dtype=torch.float32, device=dev)
    dir = torch.empty((n, 3), dtype=torch.float32, device=dev)
    c = make_cfg(cfg)
    ctx._raise(lib().pt_primary_rays(ctx.h, scene.h, C.byref(c), first_slot, n, _dptr(org), _dptr(dir),
                                     _stream(stream)))
    return org, dir


def trace_rays(ctx: Context, scene: Scene, org: torch.Tensor, dir: torch.Tensor, stream=None):
    org, dir = org.contiguous(), dir.contiguous()
    n = org.shape[0]
    t = torch.empty(n, dtype=torch.float32, device=org.device)
    prim = torch.empty(n, dtype=torch.int32, device=org.device)
    ctx._raise(lib().pt_trace_rays(ctx.h, scene.h, n, _dptr(org), _dptr(dir), _dptr(t), _dptr(prim),
                                   _stream(stream)))
    return t, prim
