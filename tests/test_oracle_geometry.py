"""Pins of the oracle's random numbers, camera and ray-primitive geometry
against published vectors, closed forms and brute force (CPU only)."""
import math
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _kat():
    rows = []
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[:4], v[4:6], v[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,want", _kat())
def test_philox_known_answers(ctr, key, want):
    assert list(O.philox(ctr, key)) == want


def test_philox_batch_matches_single_and_is_uniform():
    rng = np.random.default_rng(1)
    ctr = rng.integers(0, 2**32, size=(64, 4), dtype=np.uint64).astype(np.uint32)
    out = O.philox_batch(7, 3, ctr)
    for i in range(len(ctr)):
        assert list(out[i]) == list(O.philox(ctr[i], [7, 3]))
    # 2^16 counters -> 2^18 words; each byte value should be close to uniform
    n = 1 << 16
    c = np.zeros((n, 4), np.uint32)
    c[:, 0] = np.arange(n)
    w = O.philox_batch(0, 0, c).ravel()
    hist = np.bincount((w >> 24).astype(np.int64), minlength=256)
    exp = len(w) / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 255 + 6 * math.sqrt(2 * 255)


def test_train_uv_uses_philox_stream_one():
    uv = O.train_uv(5, 9, 8)
    for i in range(8):
        w = O.philox([i, 9, 0, 0], [5, 1])
        assert uv[i, 0] == (w[0] >> 8) / 2**24 and uv[i, 1] == (w[1] >> 8) / 2**24


# ----------------------------------------------------------------------------
def _one_sphere(c=(0, 0, 0), r=1.0):
    sc = I.furnace_sphere_outside()
    sc.sphere = np.array([[*c, r]], np.float32)
    return O.Scene(sc, use_bvh=False)


def test_sphere_closed_form_roots():
    s = _one_sphere((1.0, 2.0, -3.0), 0.5)
    # ray through the centre from distance 10: t = 10 - r
    t, ids = s.closest_hit([[1.0, 2.0, 7.0]], [[0, 0, -1.0]])
    assert ids[0] == 0 and abs(t[0] - 9.5) < 1e-12
    # tangent ray (discriminant exactly zero): touches at t = 10
    t, ids = s.closest_hit([[1.5, 2.0, 7.0]], [[0, 0, -1.0]])
    assert ids[0] == 0 and abs(t[0] - 10.0) < 1e-12
    # just outside the tangent: miss
    t, ids = s.closest_hit([[1.5 + 1e-9, 2.0, 7.0]], [[0, 0, -1.0]])
    assert ids[0] == -1 and np.isinf(t[0])
    # origin inside: exit root r - offset along the direction
    t, ids = s.closest_hit([[1.0, 2.1, -3.0]], [[0, 1.0, 0]])
    assert ids[0] == 0 and abs(t[0] - 0.4) < 1e-12
    # sphere behind the ray: miss
    t, ids = s.closest_hit([[1.0, 2.0, 7.0]], [[0, 0, 1.0]])
    assert ids[0] == -1
    # oblique ray: distance from centre to line d, t = sqrt(D^2-d^2) - sqrt(r^2-d^2)
    o = np.array([1.0 + 0.3, 2.0, 7.0])
    dirv = np.array([0.0, 0.0, -1.0])
    t, ids = s.closest_hit([o], [dirv])
    assert abs(t[0] - (10.0 - math.sqrt(0.25 - 0.09))) < 1e-12


def test_quad_hit_and_edges():
    sc = I.box_scene()
    s = O.Scene(sc, use_bvh=False)
    # straight down onto the floor (quad 0 -> global id 2) from inside the box
    t, ids = s.closest_hit([[0.4, 0.0, -0.4]], [[0, -1.0, 0]])
    assert ids[0] == 2 and abs(t[0] - 0.5) < 1e-12
    # straight up: the ceiling panel (quad 5 -> id 7) at y=0.45 is hit before the ceiling
    t, ids = s.closest_hit([[0.0, 0.0, 0.0]], [[0, 1.0, 0]])
    assert ids[0] == 7 and t[0] == float(np.float32(0.45))  # quad planes are stored as float32
    # just outside the panel: ceiling (id 3) at 0.5
    t, ids = s.closest_hit([[0.16, 0.0, 0.0]], [[0, 1.0, 0]])
    assert ids[0] == 3 and abs(t[0] - 0.5) < 1e-12
    # panel edge is inclusive
    e = float(np.float32(0.15))
    t, ids = s.closest_hit([[e, 0.0, 0.0]], [[0, 1.0, 0]])
    assert ids[0] == 7
    t, ids = s.closest_hit([[np.nextafter(e, 1.0), 0.0, 0.0]], [[0, 1.0, 0]])
    assert ids[0] == 3
    # ray along the corner edge where floor and back wall meet: equal t -> smaller id (floor=2)
    d = np.array([0.0, -1.0, -1.0]) / math.sqrt(2)
    t, ids = s.closest_hit([[0.0, 0.0, 0.0]], [d])
    assert ids[0] == 2 and abs(t[0] - 0.5 * math.sqrt(2)) < 1e-12


def _tri_cramer(v0, v1, v2, o, d):
    """Independent solve of o + t d = v0 + b1 (v1-v0) + b2 (v2-v0) (3x3 linear system)."""
    A = np.stack([-d, v1 - v0, v2 - v0], 1)
    try:
        t, b1, b2 = np.linalg.solve(A, o - v0)
    except np.linalg.LinAlgError:
        return np.inf, None
    return t, (1 - b1 - b2, b1, b2)


def test_triangle_matches_linear_solve_away_from_edges():
    rng = np.random.default_rng(3)
    sc = I.random_triangles_scene(1)
    sc.vert = np.array([[-0.7, -0.4, 0.1], [0.8, -0.5, -0.3], [0.1, 0.9, 0.2]], np.float32)
    s = O.Scene(sc, use_bvh=False)
    v = sc.vert.astype(np.float64)
    n_hit = 0
    for _ in range(3000):
        o = rng.uniform(-3, 3, 3)
        target = v.mean(0) + rng.normal(0, 0.3, 3)
        d = target - o
        d /= np.linalg.norm(d)
        t, ids = s.closest_hit([o], [d])
        tc, bary = _tri_cramer(v[0], v[1], v[2], o, d)
        inside = bary is not None and min(bary) > 1e-9 and tc > 1e-9
        outside = bary is None or min(bary) < -1e-9 or tc < -1e-9
        if inside:
            n_hit += 1
            assert ids[0] == 0 and abs(t[0] - tc) < 1e-9 * max(1, tc)
        elif outside:
            assert ids[0] == -1
    assert n_hit > 300


def test_watertight_shared_edges_and_vertices():
    """Rays aimed exactly at interior (shared) edges and vertices of a mesh
    never fall through (the Woop et al. 2013 property)."""
    N = 8
    sc = I.heightfield_scene(N)
    s = O.Scene(sc, use_bvh=True)
    v = sc.vert.astype(np.float64)
    tri = sc.tri
    edges = {}
    for t in tri:
        for a, b in ((0, 1), (1, 2), (2, 0)):
            k = (min(t[a], t[b]), max(t[a], t[b]))
            edges[k] = edges.get(k, 0) + 1
    shared = [k for k, c in edges.items() if c == 2]
    ij = np.stack(np.unravel_index(np.arange(len(v)), (N + 1, N + 1)), 1)
    interior = np.where(np.all((ij > 0) & (ij < N), 1))[0]
    rng = np.random.default_rng(4)
    misses = 0
    for k in range(2000):
        if k % 2 == 0:
            a, b = shared[rng.integers(0, len(shared))]
            lam = rng.uniform(0, 1)
            p = v[a] * (1 - lam) + v[b] * lam
        else:
            p = v[interior[rng.integers(0, len(interior))]]
        o = p + np.array([rng.uniform(-0.2, 0.2), 2.0, rng.uniform(-0.2, 0.2)])
        d = (p - o) / np.linalg.norm(p - o)
        t, ids = s.closest_hit([o], [d])
        misses += int(ids[0] < 0)
    assert misses == 0


@pytest.mark.parametrize("n_tri,n_sph,n_quad", [(200, 0, 0), (500, 40, 20), (3000, 5, 5)])
def test_bvh_equals_brute_force(n_tri, n_sph, n_quad):
    sc = I.random_triangles_scene(n_tri, seed=n_tri, n_spheres=n_sph, n_quads=n_quad)
    s = O.Scene(sc, use_bvh=True)
    rng = np.random.default_rng(5)
    o = rng.uniform(-2.5, 2.5, (2000, 3))
    d = rng.uniform(-1, 1, (2000, 3)) - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    t1, i1 = s.closest_hit(o, d, brute=False)
    t2, i2 = s.closest_hit(o, d, brute=True)
    assert np.array_equal(i1, i2)
    assert np.array_equal(t1, t2)
    assert (i1 >= 0).mean() > 0.2


def test_bvh_equals_brute_force_heightfield():
    sc = I.heightfield_scene(40, n_spheres=30)
    s = O.Scene(sc, use_bvh=True)
    org, dirs = O.primary_rays(sc.camera, 64, 64, 0, np.arange(64 * 64 * 2))
    t1, i1 = s.closest_hit(org, dirs)
    t2, i2 = s.closest_hit(org, dirs, brute=True)
    assert np.array_equal(i1, i2) and np.array_equal(t1, t2)


# ----------------------------------------------------------------------------
def test_camera_geometry():
    """Film-plane pinhole: the centre of the image looks along the view
    direction and the top edge subtends fov/2 vertically."""
    cam = I.Camera.make((1.0, 2.0, 3.0), (1.0, 2.0, -5.0), fov_deg=60.0)
    W, H = 4, 2
    # find slots whose jitter is near the pixel corner by brute-force search is
    # unnecessary: compare against the analytic direction of each slot's jitter
    slots = np.arange(W * H * 3)
    org, dirs = O.primary_rays(cam, W, H, 11, slots)
    assert np.allclose(org, [1, 2, 3])
    assert np.allclose(np.linalg.norm(dirs, axis=1), 1, atol=1e-15)
    th = math.tan(math.radians(30))
    for s, dv in zip(slots, dirs):
        pix, smp = s % (W * H), s // (W * H)
        w = O.philox([pix, smp, 0, 0], [11, 0])
        jx, jy = (w[0] >> 8) / 2**24, (w[1] >> 8) / 2**24
        fx = ((pix % W + jx) / W * 2 - 1) * th * W / H
        fy = (1 - (pix // W + jy) / H * 2) * th
        want = np.array([fx, fy, -1.0])  # camera looks down -z with up +y
        want /= np.linalg.norm(want)
        assert np.allclose(dv, want, atol=1e-14)


def test_equirect_uv_conventions():
    d = np.array([[0, 1, 0], [0, -1, 0], [0, 0, -1], [1, 0, 0], [-1, 0, 0], [0, 0, 1.0]])
    uv = O.dir_to_uv(d)
    assert abs(uv[0, 1]) < 1e-15 and abs(uv[1, 1] - 1) < 1e-15   # zenith v=0, nadir v=1
    assert np.allclose(uv[2], [0.5, 0.5]) and np.allclose(uv[3], [0.75, 0.5]) and np.allclose(uv[4], [0.25, 0.5])
    assert abs(uv[5, 0] - 1.0) < 1e-15 or abs(uv[5, 0]) < 1e-15
    # round trip with the sky generator's pixel-direction map
    rng = np.random.default_rng(0)
    th = rng.uniform(0.01, math.pi - 0.01, 100)
    ph = rng.uniform(-math.pi + 0.01, math.pi - 0.01, 100)
    dd = np.stack([np.sin(th) * np.sin(ph), np.cos(th), -np.sin(th) * np.cos(ph)], 1)
    uv = O.dir_to_uv(dd)
    assert np.allclose(uv[:, 0], 0.5 + ph / (2 * math.pi), atol=1e-13)
    assert np.allclose(uv[:, 1], th / math.pi, atol=1e-13)
