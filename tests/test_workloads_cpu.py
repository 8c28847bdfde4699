"""The seeded input recipes (CPU only): each standard workload has the shapes,
sizes and value distributions its description states, is reproducible from its
seed, and gives the field in complex64 and the heights in float64 metres."""
from __future__ import annotations

import math

import numpy as np

from paper_1203_3583_gb300 import workloads as W


def test_sinusoid64():
    g, u1, d1 = W.make("sinusoid64")
    assert (g["n1x"], g["n1y"], g["m2x"], g["m2y"]) == (64, 64, 64, 64)
    assert u1.dtype == np.complex64 and np.all(u1 == 1)
    assert d1.dtype == np.float64 and d1.shape == (64, 64)
    # 32 samples per 320 um period: the peaks reach the 20 um amplitude exactly
    assert math.isclose(d1.max(), 20e-6, rel_tol=1e-12)
    assert math.isclose(d1.min(), -20e-6, rel_tol=1e-12)
    assert np.allclose(d1, np.roll(d1, 32, axis=1)) and np.allclose(d1, np.roll(d1, 32, axis=0))


def test_spherical_cap1024():
    g, u1, d1 = W.make("spherical_cap1024")
    n, p, radius = 1024, 8e-6, 20e-3
    assert (g["n1x"], g["p1x"], g["lam"], g["z0"]) == (n, p, 532e-9, 0.2)
    # binary mask with p = 0.5, phase zero
    assert set(np.unique(u1)) <= {0, 1} and abs(np.mean(u1.real) - 0.5) < 0.01
    # zero at the corner sample (rho = half-diagonal), the cap height at the centre
    assert abs(d1[0, 0]) < 1e-15
    rho_max2 = 2 * (n / 2 * p) ** 2
    assert math.isclose(d1[n // 2, n // 2], radius - math.sqrt(radius ** 2 - rho_max2), rel_tol=1e-12)
    assert np.all(d1 >= -1e-15)


def test_smooth_random2048():
    g, u1, d1 = W.make("smooth_random2048")
    assert (g["n1x"], g["p1x"], g["lam"], g["z0"]) == (2048, 4e-6, 633e-9, 0.1)
    assert d1.min() == 0.0 and math.isclose(d1.max(), 50e-6, rel_tol=1e-12)
    amp = np.abs(u1)
    assert amp.min() >= 0.0 and amp.max() < 1.0 + 1e-6 and abs(amp.mean() - 0.5) < 0.01
    ph = np.angle(u1[amp > 0.05])
    # uniform phase: the mean unit phasor vanishes
    assert abs(np.mean(np.exp(1j * ph))) < 0.01
    # smooth: neighbouring heights differ by a small fraction of the range
    assert np.max(np.abs(np.diff(d1, axis=1))) < 0.05 * 50e-6
    g2, u2, d2 = W.make("smooth_random2048")
    assert np.array_equal(u1, u2) and np.array_equal(d1, d2)


def test_tilt_bump4096_recipe_at_reduced_size():
    g, u1, d1 = W.make("tilt_bump4096", scale=4)
    n, p = 1024, 3.74e-6
    assert (g["n1x"], g["p1x"], g["lam"], g["z0"]) == (n, p, 532e-9, 0.15)
    assert np.allclose(np.abs(u1), 1.0, atol=1e-6)
    x = (np.arange(n) - n // 2) * p
    # the centre sample carries the full 30 um bump, the row far from it the 2 degree tilt
    assert math.isclose(d1[n // 2, n // 2], 30e-6, rel_tol=1e-12)
    far = d1[0] - 30e-6 * np.exp(-(x ** 2 + (n // 2 * p) ** 2) / (2 * (2e-3) ** 2))
    assert np.allclose(far, x * math.tan(math.radians(2.0)), rtol=0, atol=1e-15)


def test_rgb_batch24():
    items = W.make_batch()
    assert len(items) == 24
    lams = [g["lam"] for g, _, _ in items]
    assert np.allclose(lams, [450e-9, 532e-9, 633e-9] * 8, rtol=1e-12, atol=0)
    for g, u1, d1 in items:
        assert g["n1x"] == g["n1y"] == g["m2x"] == g["m2y"] and g["n1x"] in (256, 512, 1024, 2048)
        assert math.isclose(g["p1x"], 3e-6) and math.isclose(g["p2x"], 3e-6)
        assert 0.05 <= g["z0"] <= 0.3
        span = d1.max() - d1.min()
        assert 5e-6 <= max(d1.max(), span / 2) <= 50e-6 + 1e-12
        assert u1.dtype == np.complex64 and u1.shape == (g["n1y"], g["n1x"])
    sizes = {g["n1x"] for g, _, _ in items}
    assert len(sizes) >= 3  # uneven sizes


def test_sample_points_distinct_and_seeded():
    g, _, _ = W.make("sinusoid64")
    mx, my = W.sample_points(g, 500, seed=9)
    assert mx.dtype == np.int32 and my.dtype == np.int32
    assert len(set(zip(mx.tolist(), my.tolist()))) == 500
    assert mx.min() >= 0 and mx.max() < 64 and my.min() >= 0 and my.max() < 64
    mx2, my2 = W.sample_points(g, 500, seed=9)
    assert np.array_equal(mx, mx2) and np.array_equal(my, my2)


def test_line_facets_layout():
    x1, d1, w = W.line_facets()
    p = 10e-6
    assert x1.size == d1.size == w.size == 1024
    # samples are the midpoints of 1024 steps of length p along the surface:
    # p apart within a segment, closer across a change of angle
    steps = np.hypot(np.diff(x1), np.diff(d1))
    assert np.all(steps <= p * (1 + 1e-12))
    # segments: flat, -30, flat, -50, flat, 0, flat, +50 degrees, 128 samples each
    ang = np.degrees(np.arctan2(np.diff(d1), np.diff(x1)))
    for k, a in enumerate((0, -30, 0, -50, 0, 0, 0, 50)):
        inner = slice(k * 128, (k + 1) * 128 - 1)
        assert np.allclose(steps[inner], p, rtol=1e-9), k
        assert np.allclose(ang[inner], a, atol=1e-9), (k, a)
        # projected weight of each sample: p |cos(angle)|
        assert np.allclose(w[k * 128:(k + 1) * 128], p * abs(math.cos(math.radians(a))), rtol=1e-12)
    assert abs(0.5 * (x1[0] + x1[-1])) < 1e-15 and abs(d1.mean()) < 1e-15


def test_line_quadratic_layout():
    x1, d1, w = W.line_quadratic()
    p = 10e-6
    assert x1.size == 1024 and np.all(np.diff(x1) > 0)
    # a parabola: constant second difference in x, 45 degree slope at the ends
    a = np.polyfit(x1, d1, 2)[0]
    assert np.allclose(d1 - d1.mean(), a * x1 ** 2 - np.mean(a * x1 ** 2), atol=1e-15)
    end_slope = 2 * a * (x1[-1] + 0.5 * w[-1])
    assert abs(end_slope - 1.0) < 0.01
    # samples p apart along the arc
    steps = np.hypot(np.diff(x1), np.diff(d1))
    assert np.allclose(steps, p, rtol=1e-3)
    assert np.allclose(w, p / np.sqrt(1 + (2 * a * x1) ** 2), rtol=1e-9)


def test_multi_surfaces():
    items = W.make_multi()
    assert [g["n1x"] for g, _, _ in items] == [384, 256, 512]
    for g, u1, d1 in items:
        assert (g["m2x"], g["m2y"], g["lam"], g["z0"]) == (1024, 1024, 532e-9, 0.2)
        assert "ox" in g and "oy" in g and u1.shape == d1.shape == (g["n1y"], g["n1x"])
    offs = {(g["ox"], g["oy"]) for g, _, _ in items}
    assert len(offs) == 3
