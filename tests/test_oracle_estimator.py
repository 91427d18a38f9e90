"""Pins of the oracle's path-tracing estimator and BSDF lobes (CPU only):
white-furnace closed forms, energy bounds, Fresnel and Snell's law."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I


@pytest.mark.parametrize("a,D", [(0.5, 5), (0.8, 3), (0.3, 1), (0.9, 8)])
def test_furnace_inside_closed_sphere(a, D):
    """Camera inside a closed Lambertian sphere with albedo a, emission 1-a:
    every path gathers (1-a) sum_{k<D} a^k = 1 - a^D, with zero variance."""
    sc = I.furnace_sphere_inside(a)
    r = O.render(O.Scene(sc), I.RenderCfg(16, 12, 3, D), want_slots=True)
    af = float(sc.mat[0, 0])          # albedo and emission as stored (float32)
    le = float(sc.mat[0, 5])
    want = le * sum(af ** k for k in range(D))
    assert np.allclose(r["slots"], want, rtol=0, atol=1e-13)
    assert abs(want - (1 - a ** D)) < 1e-6


def test_furnace_outside_convex_lambertian():
    """Convex Lambertian sphere under constant radiance 1: a path that hits
    gathers exactly a (the reflected ray escapes), a miss gathers 1."""
    a = 0.25
    sc = I.furnace_sphere_outside(a)
    r = O.render(O.Scene(sc), I.RenderCfg(24, 24, 4, 4), want_slots=True, want_ids=True)
    hit = r["ids"][:, :, 0] >= 0
    L = r["slots"]
    assert hit.mean() > 0.2 and (~hit).mean() > 0.2
    assert np.all(L[hit] == a) and np.all(L[~hit] == 1.0)
    assert np.all(r["ids"][hit][:, 1] == -1)   # second ray always escapes


def test_furnace_dielectric_paths_are_zero_or_one():
    """Dielectric weights are exactly 1: a path gathers 1 if it escapes
    within the depth limit and 0 otherwise; the pixel mean -> 1 as D grows."""
    sc = I.furnace_sphere_outside(kind=I.DIELECTRIC)
    for D, lo in [(3, 0.5), (12, 0.97)]:
        r = O.render(O.Scene(sc), I.RenderCfg(16, 16, 8, D), want_slots=True)
        L = r["slots"]
        assert np.all((L == 0.0) | (L == 1.0))
        assert L.mean() > lo


def test_furnace_rr_unbiased():
    """Russian roulette keeps the estimator's mean: 1 - a^D within 4 sigma."""
    a, D = 0.7, 8
    sc = I.furnace_sphere_inside(a)
    r = O.render(O.Scene(sc), I.RenderCfg(32, 32, 16, D, rr=True, rr_start=2), want_slots=True)
    L = r["slots"][..., 0].ravel()
    want = float(sc.mat[0, 5]) * sum(float(sc.mat[0, 0]) ** k for k in range(D))
    assert L.std() > 0  # roulette introduces variance
    assert abs(L.mean() - want) < 4 * L.std() / math.sqrt(L.size)


def test_furnace_metal_energy():
    """GGX metal with F0 = 1 under constant radiance 1: single-scattering
    energy is at most 1 and close to 1 for low roughness."""
    sc = I.furnace_sphere_outside(kind=I.METAL, f0=1.0, roughness=0.2)
    r = O.render(O.Scene(sc), I.RenderCfg(32, 32, 16, 6), want_slots=True, want_ids=True)
    hit = r["ids"][:, :, 0] >= 0
    L = r["slots"][hit][:, 0]
    m, se = L.mean(), L.std() / math.sqrt(L.size)
    assert m < 1.0 + 4 * se and m > 0.9


def _bsdf_scene():
    sc = I.furnace_sphere_outside()
    mt, m = I._mats([(I.LAMBERT, [0.4, 0.5, 0.6]), (I.METAL, [1.0, 1.0, 1.0, 0.01]),
                     (I.DIELECTRIC, [1, 1, 1, 0, 1.5]), (I.METAL, [0.5, 0.6, 0.7, 0.4])])
    sc.mat_type, sc.mat = mt, m
    return O.Scene(sc, use_bvh=False)


def test_lambert_cosine_distribution():
    s = _bsdf_scene()
    ng = np.array([0.0, 0.0, 1.0])
    d = np.array([0.3, 0.1, -1.0])
    d /= np.linalg.norm(d)
    rng = np.random.default_rng(0)
    cos = []
    for _ in range(20000):
        ok, wi, wt = O.sample_bsdf(s, 0, d, ng, rng.uniform(), rng.uniform(), 0.5)
        assert ok and np.allclose(wt, [0.4, 0.5, 0.6])
        assert abs(np.linalg.norm(wi) - 1) < 1e-14
        cos.append(wi[2])
    cos = np.array(cos)
    # cosine-weighted: E[cos] = 2/3, P(cos^2 <= x) = x
    assert cos.min() >= 0 and abs(cos.mean() - 2 / 3) < 0.01
    assert abs(np.mean(cos ** 2 <= 0.5) - 0.5) < 0.015
    # back-facing normal is flipped to the incident side
    ok, wi, _ = O.sample_bsdf(s, 0, d, -ng, 0.3, 0.3, 0.5)
    assert wi[2] > 0


def test_metal_near_mirror():
    s = _bsdf_scene()
    ng = np.array([0.0, 1.0, 0.0])
    d = np.array([1.0, -1.0, 0.0]) / math.sqrt(2)
    ok, wi, wt = O.sample_bsdf(s, 1, d, ng, 0.5, 0.25, 0.5)
    assert ok and np.allclose(wi, [1 / math.sqrt(2), 1 / math.sqrt(2), 0], atol=1e-3)
    assert np.allclose(wt, 1.0, atol=2e-3)   # F0 = 1, G -> 1 as roughness -> 0
    # Schlick at o.h = cos 45deg with F0 = (0.5, 0.6, 0.7), rough metal, h = n (u1 = 0)
    ok, wi, wt = O.sample_bsdf(s, 3, d, ng, 0.0, 0.0, 0.5)
    c = 1 / math.sqrt(2)
    f0 = np.array([0.5, 0.6, 0.7], np.float32).astype(np.float64)  # stored as float32
    alpha = float(np.float32(0.4)) ** 2
    t2 = (1 - c * c) / (c * c)
    G1 = 2 / (1 + math.sqrt(1 + alpha * alpha * t2))
    F = f0 + (1 - f0) * (1 - c) ** 5
    assert np.allclose(wi, [c, c, 0], atol=1e-12)
    assert np.allclose(wt, F * G1 * G1 * c / (c * 1.0), rtol=1e-10)


def test_dielectric_fresnel_and_snell():
    s = _bsdf_scene()
    ng = np.array([0.0, 1.0, 0.0])
    # normal incidence: F = ((1-1.5)/(1+1.5))^2 = 0.04
    d = np.array([0.0, -1.0, 0.0])
    ok, wi, wt = O.sample_bsdf(s, 2, d, ng, 0.1, 0.1, 0.0399)
    assert np.allclose(wi, [0, 1, 0]) and np.all(wt == 1.0)
    ok, wi, wt = O.sample_bsdf(s, 2, d, ng, 0.1, 0.1, 0.0401)
    assert np.allclose(wi, [0, -1, 0])
    # oblique entry: sin(theta_t) = sin(theta_i) / 1.5
    th = math.radians(50)
    d = np.array([math.sin(th), -math.cos(th), 0.0])
    ok, wi, wt = O.sample_bsdf(s, 2, d, ng, 0.1, 0.1, 0.999)
    assert wi[1] < 0 and abs(wi[0] - math.sin(th) / 1.5) < 1e-13
    # exit beyond the critical angle (asin(1/1.5) = 41.8 deg): total internal reflection
    th = math.radians(45)
    d = np.array([math.sin(th), math.cos(th), 0.0])  # travelling out through the +y face from inside
    ok, wi, wt = O.sample_bsdf(s, 2, d, ng, 0.1, 0.1, 0.999)
    assert np.allclose(wi, [math.sin(th), -math.cos(th), 0], atol=1e-14)
    # exit below the critical angle: refracts out with sin scaled by 1.5
    th = math.radians(20)
    d = np.array([math.sin(th), math.cos(th), 0.0])
    ok, wi, wt = O.sample_bsdf(s, 2, d, ng, 0.1, 0.1, 0.999)
    assert wi[1] > 0 and abs(wi[0] - 1.5 * math.sin(th)) < 1e-13
