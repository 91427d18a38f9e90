"""Seeded synthetic workloads for the neural path tracer.

This module only *creates inputs*: scene geometry, materials, cameras,
random-init network weights and a procedural HDR sky.  It holds none of the
renderer's arithmetic (no intersection, sampling, shading or network
evaluation), so both the CUDA library and the CPU oracle can consume its
arrays without sharing any method code.

The paper's own assets (Cornell-box mesh, Poly Haven HDRIs, trained NIF
weights; paper Section 4 and Appendix B) are not available, so every scene
here is a procedural stand-in shaped like the paper's five test scenes
(Fig. 1 / Table 2): a box of quads with two spheres, a field of spheres, a
small and a large BVH mesh, and the same small mesh used for radiance
caching.

Global primitive order, used for primitive IDs and tie-breaks everywhere:
spheres first, then quads, then triangles.

Material encoding (``mat`` rows): ``[albedo r, g, b, roughness, ior,
emission r, g, b]``; ``mat_type``: 0 Lambertian, 1 GGX metal, 2 dielectric.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

LAMBERT, METAL, DIELECTRIC = 0, 1, 2

# stream tags for the input generators (not the renderer's own streams)
TAG_NIF_INIT = 3
TAG_BOX_ALBEDO = 4
TAG_SKY = 5
TAG_SPHERES = 6
TAG_HEIGHTFIELD = 7
TAG_HF_SPHERES = 8


def _rng(seed: int, tag: int) -> np.random.Generator:
    return np.random.default_rng([int(seed), int(tag)])


@dataclasses.dataclass
class Camera:
    eye: np.ndarray
    target: np.ndarray
    up: np.ndarray
    fov_deg: float  # vertical field of view

    @staticmethod
    def make(eye, target, up=(0.0, 1.0, 0.0), fov_deg=45.0) -> "Camera":
        return Camera(np.asarray(eye, np.float32), np.asarray(target, np.float32),
                      np.asarray(up, np.float32), float(fov_deg))


@dataclasses.dataclass
class Scene:
    """Host arrays describing one scene (all float32 / int32, C-contiguous)."""
    sphere: np.ndarray      # [nS, 4] cx, cy, cz, r
    sphere_mat: np.ndarray  # [nS]
    quad: np.ndarray        # [nQ, 5] plane position, lo_u, hi_u, lo_v, hi_v
    quad_axis: np.ndarray   # [nQ] plane normal axis a; u = (a+1)%3, v = (a+2)%3
    quad_mat: np.ndarray    # [nQ]
    vert: np.ndarray        # [nV, 3]
    tri: np.ndarray         # [nT, 3] vertex indices
    tri_mat: np.ndarray     # [nT]
    mat_type: np.ndarray    # [nM]
    mat: np.ndarray         # [nM, 8]
    camera: Camera
    env_const: Optional[np.ndarray] = None  # [3] constant radiance, or None = NIF
    name: str = "scene"

    @property
    def n_prims(self) -> int:
        return len(self.sphere) + len(self.quad) + len(self.tri)

    @property
    def has_emission(self) -> bool:
        return bool(np.any(self.mat[:, 5:8] != 0))

    def validate(self) -> None:
        for f in ("sphere", "quad", "vert", "mat"):
            a = getattr(self, f)
            assert a.dtype == np.float32 and a.flags.c_contiguous, f
        for f in ("sphere_mat", "quad_axis", "quad_mat", "tri", "tri_mat", "mat_type"):
            a = getattr(self, f)
            assert a.dtype == np.int32 and a.flags.c_contiguous, f
        nm = len(self.mat)
        for f in ("sphere_mat", "quad_mat", "tri_mat"):
            a = getattr(self, f)
            assert a.size == 0 or (a.min() >= 0 and a.max() < nm), f


@dataclasses.dataclass
class RenderCfg:
    width: int
    height: int
    spp: int
    max_depth: int
    seed: int = 0
    rr: bool = False
    rr_start: int = 3

    @property
    def n_slots(self) -> int:
        return self.width * self.height * self.spp


@dataclasses.dataclass
class NIF:
    """HDR neural image field parameters (float32, PyTorch Linear layout).
    skip_after = s >= 1: hidden layer s (1-based) has H - 2F outputs, and
    hidden layer s + 1 takes them followed by the 2F Fourier features."""
    B: np.ndarray                 # [F, 2] Gaussian Fourier frequencies
    W: List[np.ndarray]           # per layer [out, in]
    b: List[np.ndarray]           # per layer [out]
    M: np.ndarray                 # [3, 3] fixed colour matrix applied before exp
    skip_after: int = 0           # 0: plain MLP

    @property
    def n_freq(self) -> int:
        return int(self.B.shape[0])

    @property
    def hidden(self) -> int:
        return int(self.W[-1].shape[1])   # the head's input width (the first layer may be the narrowed one)

    @property
    def n_hidden_layers(self) -> int:
        return len(self.W) - 1

    def copy(self) -> "NIF":
        return NIF(self.B.copy(), [w.copy() for w in self.W], [x.copy() for x in self.b], self.M.copy(),
                   self.skip_after)


def _empty_scene_arrays():
    return dict(
        sphere=np.zeros((0, 4), np.float32), sphere_mat=np.zeros((0,), np.int32),
        quad=np.zeros((0, 5), np.float32), quad_axis=np.zeros((0,), np.int32),
        quad_mat=np.zeros((0,), np.int32),
        vert=np.zeros((0, 3), np.float32), tri=np.zeros((0, 3), np.int32),
        tri_mat=np.zeros((0,), np.int32))


def _mats(rows: Sequence[Tuple[int, Sequence[float]]]):
    t = np.array([r[0] for r in rows], np.int32)
    m = np.zeros((len(rows), 8), np.float32)
    for i, (_, p) in enumerate(rows):
        m[i, :len(p)] = p
    return t, m


# ----------------------------------------------------------------------------
# Config 1: box of six axis-aligned quads plus two spheres
# ----------------------------------------------------------------------------
def box_scene(seed: int = 0) -> Scene:
    """Cornell-like open box [-0.5, 0.5]^3 (the +z face is open so the
    environment can light it), a small ceiling panel quad and two spheres on
    the floor.  Albedos are U[0.2, 0.8] per channel."""
    rng = _rng(seed, TAG_BOX_ALBEDO)
    n_mat = 8
    alb = rng.uniform(0.2, 0.8, size=(n_mat, 3)).astype(np.float32)
    mat_type, mat = _mats([(LAMBERT, list(alb[i])) for i in range(n_mat)])
    # axis, position, lo_u, hi_u, lo_v, hi_v with u=(a+1)%3, v=(a+2)%3
    q = [
        (1, -0.5, -0.5, 0.5, -0.5, 0.5),   # floor   y=-0.5 (u=z, v=x)
        (1, 0.5, -0.5, 0.5, -0.5, 0.5),    # ceiling y=+0.5
        (2, -0.5, -0.5, 0.5, -0.5, 0.5),   # back    z=-0.5 (u=x, v=y)
        (0, -0.5, -0.5, 0.5, -0.5, 0.5),   # left    x=-0.5 (u=y, v=z)
        (0, 0.5, -0.5, 0.5, -0.5, 0.5),    # right   x=+0.5
        (1, 0.45, -0.15, 0.15, -0.15, 0.15),  # ceiling panel y=0.45
    ]
    arr = _empty_scene_arrays()
    arr["quad_axis"] = np.array([r[0] for r in q], np.int32)
    arr["quad"] = np.array([r[1:] for r in q], np.float32)
    arr["quad_mat"] = np.arange(6, dtype=np.int32)
    arr["sphere"] = np.array([[-0.2, -0.35, -0.1, 0.15], [0.2, -0.3, 0.15, 0.2]], np.float32)
    arr["sphere_mat"] = np.array([6, 7], np.int32)
    cam = Camera.make((0.0, 0.0, 1.6), (0.0, 0.0, 0.0), fov_deg=45.0)
    return Scene(**arr, mat_type=mat_type, mat=mat, camera=cam, name="box")


# ----------------------------------------------------------------------------
# Config 2: 256 spheres with Lambertian / GGX metal / dielectric materials
# ----------------------------------------------------------------------------
def spheres_scene(n: int = 256, seed: int = 0) -> Scene:
    rng = _rng(seed, TAG_SPHERES)
    centres = rng.uniform(-10.0, 10.0, size=(n, 3))
    radii = rng.uniform(0.2, 1.5, size=(n, 1))
    kind = rng.uniform(0.0, 1.0, size=n)
    rows = []
    for i in range(n):
        if kind[i] < 0.6:
            rows.append((LAMBERT, list(rng.uniform(0.2, 0.8, 3))))
        elif kind[i] < 0.9:
            f0 = rng.uniform(0.5, 0.95, 3)
            rough = rng.uniform(0.05, 0.5)
            rows.append((METAL, [*f0, rough]))
        else:
            rows.append((DIELECTRIC, [1.0, 1.0, 1.0, 0.0, 1.5]))
    mat_type, mat = _mats(rows)
    arr = _empty_scene_arrays()
    arr["sphere"] = np.concatenate([centres, radii], 1).astype(np.float32)
    arr["sphere_mat"] = np.arange(n, dtype=np.int32)
    cam = Camera.make((0.0, 0.0, 35.0), (0.0, 0.0, 0.0), fov_deg=40.0)
    return Scene(**arr, mat_type=mat_type, mat=mat, camera=cam, name="spheres")


# ----------------------------------------------------------------------------
# Configs 3-5: fBm heightfield meshes
# ----------------------------------------------------------------------------
def _value_noise_fbm(x: np.ndarray, z: np.ndarray, seed: int, octaves: int = 6,
                     base_freq: float = 3.0, lacunarity: float = 2.0, gain: float = 0.5) -> np.ndarray:
    """fBm of lattice value noise with smoothstep interpolation, in [-1, 1]."""
    rng = _rng(seed, TAG_HEIGHTFIELD)
    total = np.zeros_like(x, dtype=np.float64)
    amp, norm, freq = 1.0, 0.0, base_freq
    for _ in range(octaves):
        n_cells = int(math.ceil(2.0 * freq)) + 2
        lat = rng.uniform(-1.0, 1.0, size=(n_cells + 1, n_cells + 1))
        gx = (x + 1.0) * freq
        gz = (z + 1.0) * freq
        ix = np.clip(np.floor(gx).astype(np.int64), 0, n_cells - 1)
        iz = np.clip(np.floor(gz).astype(np.int64), 0, n_cells - 1)
        fx = gx - ix
        fz = gz - iz
        sx = fx * fx * (3.0 - 2.0 * fx)
        sz = fz * fz * (3.0 - 2.0 * fz)
        a = lat[ix, iz] * (1 - sx) + lat[ix + 1, iz] * sx
        b = lat[ix, iz + 1] * (1 - sx) + lat[ix + 1, iz + 1] * sx
        total += amp * (a * (1 - sz) + b * sz)
        norm += amp
        amp *= gain
        freq *= lacunarity
    return total / norm


def heightfield_scene(n_cells: int, n_spheres: int = 0, seed: int = 0,
                      env_const: Optional[Sequence[float]] = None, name: str = "heightfield") -> Scene:
    """Heightfield over [-1, 1]^2 in x-z with height 0.2 * fBm, N+1 by N+1
    vertices, two triangles per cell split along a fixed diagonal.
    ``n_spheres`` small Lambertian spheres (r ~ U[0.005, 0.03]) sit on it."""
    N = int(n_cells)
    g = np.linspace(-1.0, 1.0, N + 1)
    X, Z = np.meshgrid(g, g, indexing="ij")  # X[i, j] = g[i], Z[i, j] = g[j]
    Y = 0.2 * _value_noise_fbm(X, Z, seed)
    vert = np.stack([X, Y, Z], -1).reshape(-1, 3).astype(np.float32)
    i = np.arange(N)
    I, J = np.meshgrid(i, i, indexing="ij")
    v00 = (I * (N + 1) + J).ravel()
    v10 = ((I + 1) * (N + 1) + J).ravel()
    v01 = (I * (N + 1) + J + 1).ravel()
    v11 = ((I + 1) * (N + 1) + J + 1).ravel()
    tri = np.empty((2 * N * N, 3), np.int64)
    tri[0::2] = np.stack([v00, v01, v11], 1)
    tri[1::2] = np.stack([v00, v11, v10], 1)
    rng = _rng(seed, TAG_HF_SPHERES)
    rows = [(LAMBERT, list(rng.uniform(0.3, 0.7, 3)))]
    arr = _empty_scene_arrays()
    arr["vert"] = vert
    arr["tri"] = tri.astype(np.int32)
    arr["tri_mat"] = np.zeros((len(tri),), np.int32)
    if n_spheres:
        sx = rng.uniform(-0.95, 0.95, n_spheres)
        sz = rng.uniform(-0.95, 0.95, n_spheres)
        sr = rng.uniform(0.005, 0.03, n_spheres)
        sy = 0.2 * _value_noise_fbm(sx, sz, seed) + sr
        arr["sphere"] = np.stack([sx, sy, sz, sr], 1).astype(np.float32)
        for _ in range(n_spheres):
            rows.append((LAMBERT, list(rng.uniform(0.3, 0.7, 3))))
        arr["sphere_mat"] = np.arange(1, n_spheres + 1, dtype=np.int32)
    mat_type, mat = _mats(rows)
    cam = Camera.make((0.0, 0.8, 1.6), (0.0, 0.0, 0.0), fov_deg=50.0)
    env = None if env_const is None else np.asarray(env_const, np.float32)
    return Scene(**arr, mat_type=mat_type, mat=mat, camera=cam, env_const=env, name=name)


# ----------------------------------------------------------------------------
# Closed-form test scenes (white furnace) and tiny triangle scenes
# ----------------------------------------------------------------------------
def furnace_sphere_outside(albedo: float = 0.5, kind: int = LAMBERT, f0: float = 1.0,
                           roughness: float = 0.3) -> Scene:
    """One unit sphere at the origin under constant radiance 1, camera outside."""
    if kind == LAMBERT:
        mt, m = _mats([(LAMBERT, [albedo] * 3)])
    elif kind == METAL:
        mt, m = _mats([(METAL, [f0] * 3 + [roughness])])
    else:
        mt, m = _mats([(DIELECTRIC, [1.0, 1.0, 1.0, 0.0, 1.5])])
    arr = _empty_scene_arrays()
    arr["sphere"] = np.array([[0.0, 0.0, 0.0, 1.0]], np.float32)
    arr["sphere_mat"] = np.zeros(1, np.int32)
    cam = Camera.make((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), fov_deg=40.0)
    return Scene(**arr, mat_type=mt, mat=m, camera=cam, env_const=np.ones(3, np.float32), name="furnace_out")


def furnace_sphere_inside(albedo: float = 0.5) -> Scene:
    """Camera inside a closed Lambertian sphere of albedo a emitting 1 - a."""
    mt, m = _mats([(LAMBERT, [albedo] * 3 + [0.0, 0.0] + [1.0 - albedo] * 3)])
    arr = _empty_scene_arrays()
    arr["sphere"] = np.array([[0.0, 0.0, 0.0, 2.0]], np.float32)
    arr["sphere_mat"] = np.zeros(1, np.int32)
    cam = Camera.make((0.1, -0.2, 0.3), (0.0, 0.0, -1.0), fov_deg=60.0)
    return Scene(**arr, mat_type=mt, mat=m, camera=cam, env_const=np.zeros(3, np.float32), name="furnace_in")


def random_triangles_scene(n_tri: int, seed: int = 0, n_spheres: int = 0, n_quads: int = 0) -> Scene:
    """Random triangle soup (plus optional spheres and quads) in [-1, 1]^3."""
    rng = np.random.default_rng([seed, 99])
    c = rng.uniform(-1, 1, size=(n_tri, 1, 3))
    v = (c + rng.normal(0, 0.15, size=(n_tri, 3, 3))).reshape(-1, 3).astype(np.float32)
    arr = _empty_scene_arrays()
    arr["vert"] = v
    arr["tri"] = np.arange(3 * n_tri, dtype=np.int32).reshape(-1, 3)
    arr["tri_mat"] = np.zeros(n_tri, np.int32)
    if n_spheres:
        arr["sphere"] = np.concatenate([rng.uniform(-1, 1, (n_spheres, 3)),
                                        rng.uniform(0.05, 0.3, (n_spheres, 1))], 1).astype(np.float32)
        arr["sphere_mat"] = np.zeros(n_spheres, np.int32)
    if n_quads:
        ax = rng.integers(0, 3, n_quads).astype(np.int32)
        pos = rng.uniform(-1, 1, n_quads)
        lo = rng.uniform(-1, 0.5, (n_quads, 2))
        hi = lo + rng.uniform(0.1, 0.5, (n_quads, 2))
        arr["quad"] = np.stack([pos, lo[:, 0], hi[:, 0], lo[:, 1], hi[:, 1]], 1).astype(np.float32)
        arr["quad_axis"] = ax
        arr["quad_mat"] = np.zeros(n_quads, np.int32)
    mt, m = _mats([(LAMBERT, [0.5, 0.5, 0.5])])
    cam = Camera.make((0.0, 0.0, 3.0), (0.0, 0.0, 0.0), fov_deg=50.0)
    return Scene(**arr, mat_type=mt, mat=m, camera=cam, env_const=np.ones(3, np.float32), name="tris")


# ----------------------------------------------------------------------------
# Neural image field weights and the procedural HDR sky
# ----------------------------------------------------------------------------
YUV_TO_RGB_BT601 = np.array([[1.0, 0.0, 1.13983],
                             [1.0, -0.39465, -0.58060],
                             [1.0, 2.03211, 0.0]], np.float32)
# YCoCg -> RGB (R = Y + Co - Cg, G = Y + Cg, B = Y - Co - Cg): the network's three outputs are (Y, Co, Cg)
YCOCG_TO_RGB = np.array([[1.0, 1.0, -1.0], [1.0, 0.0, 1.0], [1.0, -1.0, -1.0]], np.float32)


def paper_skip_layer(n_hidden_layers: int) -> int:
    """The 1-based hidden layer whose output the paper concatenates with the
    Fourier features: the last odd layer (0-based) before the middle of the
    network; 0 when there is none (fewer than three hidden layers)."""
    odd = [i for i in range(n_hidden_layers) if i % 2 == 1 and i < n_hidden_layers / 2]
    return odd[-1] + 1 if odd else 0


def nif_init(n_freq: int = 64, hidden: int = 128, n_hidden_layers: int = 3, sigma: float = 10.0,
             seed: int = 0, colour: str = "identity", skip_after: int = 0) -> NIF:
    """Random-init NIF: Fourier matrix entries N(0, sigma^2), weights
    N(0, 1/fan_in), zero biases.  Layer widths: 2F -> H (x L) -> 3; with
    skip_after = s, hidden layer s has H - 2F outputs and layer s + 1 takes
    them with the 2F features appended."""
    rng = _rng(seed, TAG_NIF_INIT)
    B = rng.normal(0.0, sigma, size=(n_freq, 2)).astype(np.float32)
    assert 0 <= skip_after < n_hidden_layers and (skip_after == 0 or hidden > 2 * n_freq)
    dims = [2 * n_freq] + [hidden] * n_hidden_layers + [3]
    W, b = [], []
    for i in range(len(dims) - 1):
        fan_in, fan_out = dims[i], dims[i + 1]
        if skip_after and i == skip_after - 1:
            fan_out = hidden - 2 * n_freq
        W.append(rng.normal(0.0, 1.0 / math.sqrt(fan_in), size=(fan_out, fan_in)).astype(np.float32))
        b.append(np.zeros((fan_out,), np.float32))
    if colour == "identity":
        M = np.eye(3, dtype=np.float32)
    elif colour == "ycocg":
        M = YCOCG_TO_RGB.copy()
    else:
        M = YUV_TO_RGB_BT601.copy()
    return NIF(B, W, b, M, skip_after)


def procedural_sky(width: int = 2048, height: int = 1024, seed: int = 0) -> np.ndarray:
    """HDR equirectangular sky [height, width, 3] float32: zenith-to-horizon
    gradient, dim ground, a sun disk of radiance 1e4 at elevation 40 deg /
    azimuth 60 deg (angular radius 1 deg) and three Gaussian lobes.

    Row 0 is the zenith (v = 0); u = 0.5 + atan2(dx, -dz) / (2 pi)."""
    rng = _rng(seed, TAG_SKY)
    v = (np.arange(height) + 0.5) / height
    u = (np.arange(width) + 0.5) / width
    U, V = np.meshgrid(u, v)  # [H, W]
    theta = V * math.pi
    phi = (U - 0.5) * 2.0 * math.pi
    d = np.stack([np.sin(theta) * np.sin(phi), np.cos(theta), -np.sin(theta) * np.cos(phi)], -1)
    zen = np.array([0.6, 1.0, 2.0])
    hor = np.array([1.0, 0.95, 0.9])
    t = np.clip(V / 0.5, 0.0, 1.0)[..., None]
    sky = zen * (1 - t) + hor * t
    ground = 0.2 * np.array([0.6, 0.5, 0.4])
    sky = np.where((V >= 0.5)[..., None], ground, sky)
    el, az = math.radians(40.0), math.radians(60.0)
    ts = math.pi / 2 - el
    sun = np.array([math.sin(ts) * math.sin(az), math.cos(ts), -math.sin(ts) * math.cos(az)])
    cosang = d @ sun
    sky = sky + (cosang >= math.cos(math.radians(1.0)))[..., None] * (1e4 * np.array([1.0, 0.95, 0.85]))
    for _ in range(3):
        cu, cv = rng.uniform(0, 1), rng.uniform(0.1, 0.45)
        sig = rng.uniform(0.02, 0.1)
        amp = rng.uniform(2.0, 20.0)
        col = rng.uniform(0.5, 1.0, 3)
        du = np.abs(U - cu)
        du = np.minimum(du, 1.0 - du)
        g = np.exp(-(du ** 2 + (V - cv) ** 2) / (2 * sig ** 2))
        sky = sky + amp * g[..., None] * col
    return np.ascontiguousarray(sky.astype(np.float32))


TAG_CACHE_INIT = 9


@dataclasses.dataclass
class CacheNet:
    """Neural radiance cache parameters (float32, PyTorch Linear layout):
    J frequencies per position axis, hidden width H, L hidden layers, and
    the box [lo, hi] that positions are normalised to."""
    n_freq: int
    W: List[np.ndarray]
    b: List[np.ndarray]
    lo: np.ndarray
    hi: np.ndarray

    @property
    def hidden(self) -> int:
        return int(self.W[0].shape[0])

    @property
    def n_hidden_layers(self) -> int:
        return len(self.W) - 1

    @property
    def in_dim(self) -> int:
        return 6 * self.n_freq + 6

    def copy(self) -> "CacheNet":
        return CacheNet(self.n_freq, [w.copy() for w in self.W], [x.copy() for x in self.b], self.lo.copy(),
                        self.hi.copy())


def scene_bounds(scene: Scene) -> Tuple[np.ndarray, np.ndarray]:
    """Axis-aligned float32 bounds of every primitive of a scene."""
    lo = np.full(3, np.inf, np.float32)
    hi = np.full(3, -np.inf, np.float32)
    if len(scene.sphere):
        lo = np.minimum(lo, (scene.sphere[:, :3] - scene.sphere[:, 3:]).min(0))
        hi = np.maximum(hi, (scene.sphere[:, :3] + scene.sphere[:, 3:]).max(0))
    if len(scene.tri):
        used = scene.vert[np.unique(scene.tri)]
        lo = np.minimum(lo, used.min(0))
        hi = np.maximum(hi, used.max(0))
    for i in range(len(scene.quad)):
        a = scene.quad_axis[i]
        u, v = (a + 1) % 3, (a + 2) % 3
        p = scene.quad[i]
        qlo = np.zeros(3, np.float32)
        qhi = np.zeros(3, np.float32)
        qlo[a] = qhi[a] = p[0]
        qlo[u], qhi[u], qlo[v], qhi[v] = p[1], p[2], p[3], p[4]
        lo, hi = np.minimum(lo, qlo), np.maximum(hi, qhi)
    return lo.astype(np.float32), hi.astype(np.float32)


def cache_init(lo, hi, n_freq: int = 12, hidden: int = 64, n_hidden_layers: int = 5, seed: int = 0) -> CacheNet:
    """Random-init radiance cache: W ~ N(0, 1/fan_in), zero biases."""
    rng = _rng(seed, TAG_CACHE_INIT)
    dims = [6 * n_freq + 6] + [hidden] * n_hidden_layers + [3]
    W, b = [], []
    for i in range(len(dims) - 1):
        W.append(rng.normal(0.0, 1.0 / math.sqrt(dims[i]), size=(dims[i + 1], dims[i])).astype(np.float32))
        b.append(np.zeros((dims[i + 1],), np.float32))
    return CacheNet(n_freq, W, b, np.asarray(lo, np.float32), np.asarray(hi, np.float32))


# ----------------------------------------------------------------------------
# The five workload configurations
# ----------------------------------------------------------------------------
CONFIGS = {
    "C1": dict(desc="box: 6 quads + 2 spheres, 64x64, 8 spp, depth 4, random-init FP32 NIF",
               cfg=RenderCfg(64, 64, 8, 4)),
    "C2": dict(desc="256 spheres + HDR-NIF, 512x512, 64 spp, depth 8",
               cfg=RenderCfg(512, 512, 64, 8)),
    "C3": dict(desc="heightfield 2x224x224 tris + HDR-NIF, 1024x1024, 16 spp, depth 6",
               cfg=RenderCfg(1024, 1024, 16, 6)),
    "C4": dict(desc="heightfield 2x2236x2236 tris + 1000 spheres, constant env, 1920x1080, 32 spp, depth 8",
               cfg=RenderCfg(1920, 1080, 32, 8)),
    "C5": dict(desc="radiance cache on the C3 scene, 1024x1024, 4 spp, 60 frames",
               cfg=RenderCfg(1024, 1024, 4, 6)),
}


def make_scene(config: str, seed: int = 0) -> Scene:
    if config == "C1":
        return box_scene(seed)
    if config == "C2":
        return spheres_scene(256, seed)
    if config in ("C3", "C5"):
        return heightfield_scene(224, 0, seed, name="small_bvh")
    if config == "C4":
        return heightfield_scene(2236, 1000, seed, env_const=(1.0, 1.0, 1.0), name="large_bvh")
    raise KeyError(config)


def uniform_uv(n: int, seed: int = 0) -> np.ndarray:
    """n uniform (u, v) pairs in [0, 1)^2 (float32 [n, 2]) for standalone NIF tests."""
    return _rng(seed, 11).uniform(0.0, 1.0, size=(n, 2)).astype(np.float32)
