"""Pins of the oracle's GGX metal lobe (CPU only) against an independent
quadrature of the microfacet BRDF (Walter, Marschner, Li, Torrance 2007).

The oracle samples a half vector h from the GGX distribution D (its
inverse CDF in tan^2), reflects the outgoing direction about h, and weights
the sample F G (o.h) / ((n.o)(n.h)).  The expected weight is therefore the
directional albedo

    E(o) = integral over the hemisphere of f(o, i) (n.i) d omega_i,
    f = D(h) G1(o) G1(i) F(o.h) / (4 (n.o)(n.i)),

which this file evaluates without the sampler: with d omega_i =
4 (o.h) d omega_h it becomes an integral of D(h) G1(o) G1(i) F(o.h) (o.h) /
(n.o) over half vectors, computed by composite Gauss-Legendre in theta_h
(panels graded around alpha, where D is concentrated) and the midpoint rule
in phi_h.  D and G1 are written here from Walter et al.'s definitions (GGX
normal distribution, Smith G1 of the GGX slope distribution), Schlick's F
with F0 = albedo, alpha = roughness^2 (the material reading of the method's
scenes).

The sampler's mean is taken as a quadrature in sample space too (graded
Gauss-Legendre in u1 towards 1, where the GGX tail lives; midpoint in u2),
so the two sides agree to ~3e-5 and the tolerance is 1e-4.  A second test
bins the sampled cos(theta_h) at normal incidence against the probability
of each bin under D(h) cos(theta_h) (chi-square).

What these pins catch, recorded by test_variants_are_far_outside_tolerance:
drawing h with alpha = roughness instead of roughness^2 (an alpha / alpha^2
slip in the sampler's tan^2), and dropping the masking term (G1 = 1), each
move the albedo by far more than the tolerance at roughness 0.2 and 0.5.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2305_20061_gb300 import inputs as I

ROUGH = (0.05, 0.2, 0.5)
F0S = (1.0, 0.5)
THETA_O = (0.0, 45.0, 75.0)
TOL = 1e-4


def _gl(edges, k):
    x, w = np.polynomial.legendre.leggauss(k)
    xs, ws = [], []
    for a, b in zip(edges[:-1], edges[1:]):
        xs.append(0.5 * (b - a) * x + 0.5 * (a + b))
        ws.append(0.5 * (b - a) * w)
    return np.concatenate(xs), np.concatenate(ws)


def _theta_nodes(alpha):
    """Panels graded geometrically from alpha / 64, plus a panel edge at 45
    degrees (where reflection about h leaves the hemisphere at normal
    incidence)."""
    edges, t = [0.0], alpha / 64
    while t < math.pi / 2:
        edges.append(t)
        t *= 1.5
    edges += [math.pi / 4, math.pi / 2]
    return _gl(np.unique(edges), 24)


def ggx_D(theta_h, alpha):
    """GGX normal distribution (Walter et al. 2007, Eq. 33)."""
    c2 = np.cos(theta_h) ** 2
    t2 = np.tan(theta_h) ** 2
    return alpha * alpha / (math.pi * c2 * c2 * (alpha * alpha + t2) ** 2)


def smith_G1(cos_v, alpha):
    """Smith shadowing of the GGX slope distribution (Walter et al. 2007, Eq. 34)."""
    t2 = (1.0 - cos_v ** 2) / cos_v ** 2
    return 2.0 / (1.0 + np.sqrt(1.0 + alpha * alpha * t2))


def albedo_quadrature(theta_o, alpha, f0, d_alpha=None, masking=True, n_phi=2048):
    """Directional albedo of the GGX metal seen from theta_o (n = +z),
    integrated over half vectors.  d_alpha replaces alpha in D only and
    masking=False sets G1 = 1: the two variants of the sampler that the
    pins must be able to tell apart."""
    d_alpha = alpha if d_alpha is None else d_alpha
    th, wth = _theta_nodes(min(alpha, d_alpha))
    phi = (np.arange(n_phi) + 0.5) * (2 * math.pi / n_phi)
    TH, PH = np.meshgrid(th, phi, indexing="ij")
    h = np.stack([np.sin(TH) * np.cos(PH), np.sin(TH) * np.sin(PH), np.cos(TH)], -1)
    o = np.array([math.sin(theta_o), 0.0, math.cos(theta_o)])
    oh = h @ o
    wi = 2.0 * oh[..., None] * h - o
    ni, no = wi[..., 2], o[2]
    valid = (oh > 0) & (ni > 0)
    F = f0 + (1.0 - f0) * (1.0 - np.clip(oh, 0.0, 1.0)) ** 5
    G = smith_G1(no, alpha) * smith_G1(np.where(valid, ni, 1.0), alpha) if masking else 1.0
    f = np.where(valid, ggx_D(TH, d_alpha) * F * G * oh / no * np.sin(TH), 0.0)
    return float((f * wth[:, None]).sum() * (2 * math.pi / n_phi))


@pytest.fixture(scope="module")
def metals():
    sc = I.furnace_sphere_outside()
    rows = [(I.METAL, [f0, f0, f0, r]) for r in ROUGH for f0 in F0S]
    sc.mat_type, sc.mat = I._mats(rows)
    return O.Scene(sc, use_bvh=False), sc.mat


def _sample_space_nodes():
    """(u1, u2) nodes and weights of a quadrature over the unit square:
    Gauss-Legendre in u1 on panels [1 - 2^-k, 1 - 2^-(k+1)] (the tail of
    tan^2 = alpha^2 u1 / (1 - u1) lies at u1 -> 1), midpoint in u2."""
    edges = np.array([0.0] + [1.0 - 2.0 ** -k for k in range(1, 31)] + [1.0])
    x1, w1 = _gl(edges, 16)
    n2 = 1024
    x2 = (np.arange(n2) + 0.5) / n2
    U1, U2 = np.meshgrid(x1, x2, indexing="ij")
    W = np.outer(w1, np.full(n2, 1.0 / n2)).ravel()
    return np.stack([U1.ravel(), U2.ravel(), np.full(U1.size, 0.5)], 1), W


def test_metal_albedo_matches_microfacet_quadrature(metals):
    """Mean sample weight of the oracle's GGX lobe = directional albedo of
    the microfacet BRDF, for roughness 0.05 / 0.2 / 0.5, F0 = 1 / 0.5 and
    incidence 0 / 45 / 75 degrees (every channel carries the same F0)."""
    osc, mat = metals
    u, W = _sample_space_nodes()
    ng = np.array([0.0, 0.0, 1.0])
    for mi in range(len(mat)):
        alpha = float(mat[mi, 3]) ** 2          # roughness as stored (float32), squared
        f0 = float(mat[mi, 0])
        for th in THETA_O:
            tho = math.radians(th)
            d = -np.array([math.sin(tho), 0.0, math.cos(tho)])
            ok, wi, wt = O.sample_bsdf_batch(osc, mi, d, ng, u)
            assert np.all(wt[ok] >= 0) and np.all(wt[~ok] == 0)
            assert np.allclose(np.linalg.norm(wi[ok], axis=1), 1.0, atol=1e-12)
            assert np.all(wi[ok][:, 2] > 0)
            mean = float((wt[:, 0] * W).sum())
            want = albedo_quadrature(tho, alpha, f0)
            assert abs(mean - want) <= TOL, (float(mat[mi, 3]), f0, th, mean, want)


@pytest.mark.parametrize("rough", ROUGH)
def test_half_vector_distribution_chi_square(metals, rough):
    """At normal incidence h = normalize(o + i) of each valid sample is
    distributed as D(h) cos(theta_h); samples with theta_h > 45 degrees
    reflect below the horizon and are absorbed.  Twenty bins of equal
    probability (edges from the quadrature's CDF) plus the absorbed bin,
    2^20 random (u1, u2)."""
    from scipy import stats
    osc, mat = metals
    mi = ROUGH.index(rough) * len(F0S)
    alpha = float(mat[mi, 3]) ** 2
    # CDF of theta_h under D cos sin (2 pi) on a fine graded grid
    th = np.concatenate([[0.0], np.geomspace(alpha / 256, math.pi / 2, 20000)])
    mid = 0.5 * (th[1:] + th[:-1])
    dens = 2 * math.pi * ggx_D(mid, alpha) * np.cos(mid) * np.sin(mid) * np.diff(th)
    cdf = np.concatenate([[0.0], np.cumsum(dens)])
    assert abs(cdf[-1] - 1.0) < 1e-4                    # D cos(theta_h) is normalised
    p45 = float(np.interp(math.pi / 4, th, cdf))
    nb = 20
    edges = np.interp(np.linspace(0, p45, nb + 1), cdf, th)
    edges[0], edges[-1] = 0.0, math.pi / 4
    expect = np.append(np.diff(np.interp(edges, th, cdf)), 1.0 - p45)
    rng = np.random.default_rng(7)
    n = 1 << 20
    u = np.stack([rng.uniform(size=n), rng.uniform(size=n), np.full(n, 0.5)], 1)
    ok, wi, _ = O.sample_bsdf_batch(osc, mi, np.array([0.0, 0.0, -1.0]), np.array([0.0, 0.0, 1.0]), u)
    h = wi[ok] + np.array([0.0, 0.0, 1.0])
    th_h = np.arccos(np.clip(h[:, 2] / np.linalg.norm(h, axis=1), -1, 1))
    counts = np.append(np.histogram(th_h, bins=edges)[0], (~ok).sum())
    chi2 = float(((counts - n * expect) ** 2 / (n * expect)).sum())
    assert stats.chi2.sf(chi2, nb) > 1e-3, (chi2, counts, n * expect)


def test_variants_are_far_outside_tolerance():
    """The mistakes the albedo pin exists to catch move the albedo by far
    more than TOL: h drawn with alpha = roughness (alpha / alpha^2 slip) and
    G1 = 1 (masking dropped)."""
    worst_swap = worst_mask = 0.0
    for r in (0.2, 0.5):
        alpha = r * r
        for th in THETA_O:
            tho = math.radians(th)
            ref = albedo_quadrature(tho, alpha, 1.0)
            worst_swap = max(worst_swap, abs(albedo_quadrature(tho, alpha, 1.0, d_alpha=r) - ref))
            worst_mask = max(worst_mask, abs(albedo_quadrature(tho, alpha, 1.0, masking=False) - ref))
    assert worst_swap > 100 * TOL and worst_mask > 100 * TOL, (worst_swap, worst_mask)
    # even the near-mirror lobe separates the alpha slip
    ref = albedo_quadrature(0.0, 0.05 ** 2, 1.0)
    assert abs(albedo_quadrature(0.0, 0.05 ** 2, 1.0, d_alpha=0.05) - ref) > 10 * TOL


def test_quadrature_closed_forms():
    """The quadrature itself, against closed forms: D cos(theta_h) integrates
    to 1 over the hemisphere, and with G1 = 1, F0 = 1 at normal incidence
    the albedo is the probability that theta_h < 45 degrees,
    1 / (1 + alpha^2) for GGX (its CDF in tan^2 is x / (alpha^2 + x))."""
    for alpha in (0.05 ** 2, 0.04, 0.25, 0.7):
        th, w = _theta_nodes(alpha)
        assert abs(float((2 * math.pi * ggx_D(th, alpha) * np.cos(th) * np.sin(th) * w).sum()) - 1.0) < 1e-9
        e = albedo_quadrature(0.0, alpha, 1.0, masking=False, n_phi=64)
        assert abs(e - 1.0 / (1.0 + alpha * alpha)) < 1e-9, (alpha, e)
