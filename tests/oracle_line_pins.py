"""Pins of the 1D oracle (oracle/line.py): closed forms, identities and
limits that fix the one-dimensional Eq. 7 / 5 / 2 with explicit samples.
Each pin returns an error to compare with its tolerance in LINE_PINS.
Shared by test_oracle_line_pins.py (against the oracle and planted mistakes)."""
from __future__ import annotations

import numpy as np


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def _uniform(n, p):
    return (np.arange(n) - n // 2) * p


def _field(rng, n):
    return rng.standard_normal(n) + 1j * rng.standard_normal(n)


def pin_fft_natural_pitch(line, n=48, p1=10e-6, lam=633e-9, z0=0.05, seed=41):
    """Uniform samples x1 = (n - N/2) p1, d1 = 0, w = p1, and p2 = lambda z0/(N p1):
    the sum is a centred DFT of u1 exp(ik x1^2/(2 z0)) (numpy's FFT)."""
    rng = np.random.default_rng(seed)
    u1 = _field(rng, n)
    x1 = _uniform(n, p1)
    p2 = lam * z0 / (n * p1)
    k = 2 * np.pi / lam
    f = u1 * np.exp(1j * k * x1 ** 2 / (2 * z0))
    dft = np.fft.fftshift(np.fft.fft(np.fft.ifftshift(f)))
    x2 = _uniform(n, p2)
    ref = np.exp(1j * k * (z0 + x2 ** 2 / (2 * z0))) / np.sqrt(1j * lam * z0) * p1 * dft
    g = dict(m2=n, p2=p2, lam=lam, z0=z0)
    return rel_l2(line(g, x1, np.zeros(n), np.full(n, p1), u1, 7), ref)


def pin_planar_shift(line, c=0.3e-3, n=40, p1=9e-6, m2=36, p2=11e-6, lam=532e-9, z0=0.04,
                     s=0.013, seed=42):
    """d1 = c with a tilted incident wave: Eq. 7 equals sqrt(r0/z0) exp(ikc)
    exp(ik c (sz - 1)) exp(ik x2^2 (1/z0 - 1/r0)/2) times Eq. 7 of the flat
    source at distance r0 = z0 - c."""
    rng = np.random.default_rng(seed)
    u1 = _field(rng, n)
    x1 = _uniform(n, p1) + 0.3 * p1 * rng.standard_normal(n)  # non-uniform positions
    w = np.full(n, p1)
    r0 = z0 - c
    k = 2 * np.pi / lam
    sz = np.sqrt(1 - s ** 2)
    x2 = _uniform(m2, p2)
    g = dict(m2=m2, p2=p2, lam=lam, z0=z0, s=s)
    ref = (line(dict(g, z0=r0), x1, np.zeros(n), w, u1, 7) * np.sqrt(r0 / z0)
           * np.exp(1j * k * c * sz) * np.exp(1j * k * x2 ** 2 * (1 / z0 - 1 / r0) / 2))
    return rel_l2(line(g, x1, np.full(n, c), w, u1, 7), ref)


def pin_gaussian(line, c=0.2e-3, n=256, p1=10e-6, m2=40, p2=11e-6, lam=633e-9, z0=0.05,
                 s=0.002):
    """Gaussian u1 = exp(-x1^2/w0^2) on d1 = c, lit at direction cosine s:
    with a = 1/w0^2 - ik/(2 r0) the integral of u1 exp(ik x1^2/(2 r0))
    exp(-ik x1 (x2 - r0 s)/r0) is sqrt(pi/a) exp(-(k (x2 - r0 s)/r0)^2/(4a))."""
    k = 2 * np.pi / lam
    w0 = n * p1 / 10
    x1 = _uniform(n, p1)
    u1 = np.exp(-x1 ** 2 / w0 ** 2).astype(np.complex128)
    r0 = z0 - c
    sz = np.sqrt(1 - s ** 2)
    a = 1 / w0 ** 2 - 1j * k / (2 * r0)
    x2 = _uniform(m2, p2)
    integral = np.sqrt(np.pi / a) * np.exp(-(k * (x2 - r0 * s) / r0) ** 2 / (4 * a))
    ref = (np.exp(1j * k * (z0 + x2 ** 2 / (2 * z0))) / np.sqrt(1j * lam * z0)
           * np.exp(1j * k * c * (sz - 1)) * integral)
    g = dict(m2=m2, p2=p2, lam=lam, z0=z0, s=s)
    return rel_l2(line(g, x1, np.full(n, c), np.full(n, p1), u1, 7), ref)


def pin_permute_and_split(line, n=30, lam=633e-9, z0=0.05, seed=43):
    """The sum does not depend on the order of the samples, and a sample of
    weight w equals two samples of weight w/2 at the same place (forms 7, 5, 2)."""
    rng = np.random.default_rng(seed)
    x1 = rng.uniform(-200e-6, 200e-6, n)
    d1 = rng.uniform(-50e-6, 50e-6, n)
    w = rng.uniform(5e-6, 15e-6, n)
    u1 = _field(rng, n)
    g = dict(m2=24, p2=12e-6, lam=lam, z0=z0, s=-0.01)
    perm = rng.permutation(n)
    err = 0.0
    for form in (7, 5, 2):
        ref = line(g, x1, d1, w, u1, form)
        err = max(err, rel_l2(line(g, x1[perm], d1[perm], w[perm], u1[perm], form), ref))
        x2_, d2_, w2_, u2_ = (np.concatenate([x1, x1[:5]]), np.concatenate([d1, d1[:5]]),
                              np.concatenate([w, w[:5] / 2]), np.concatenate([u1, u1[:5]]))
        w2_[:5] /= 2
        err = max(err, rel_l2(line(g, x2_, d2_, w2_, u2_, form), ref))
    return err


def pin_eq5_equals_eq7_flat(line, n=36, lam=633e-9, z0=0.05, seed=44):
    """d1 = 0: r0 = z0 for every sample, so Eq. 6 is exact and Eq. 5 is Eq. 7."""
    rng = np.random.default_rng(seed)
    x1 = np.sort(rng.uniform(-150e-6, 150e-6, n))
    u1 = _field(rng, n)
    g = dict(m2=20, p2=10e-6, lam=lam, z0=z0, s=0.01)
    w = np.full(n, 8e-6)
    return rel_l2(line(g, x1, np.zeros(n), w, u1, 5), line(g, x1, np.zeros(n), w, u1, 7))


def pin_eq5_planar_shift(line, c=0.35e-3, n=34, lam=532e-9, z0=0.04, s=0.012, seed=47):
    """d1 = c: the exponentials of Eq. 5 combine to exp(ik s x1) exp(ik c (sz - 1))
    exp(ik (x1 - x2)^2/(2 r0)), planar Fresnel propagation over r0 = z0 - c
    with the prefactor of z0: Eq. 5 = sqrt(r0/z0) exp(ik sz c) Eq. 7(r0, d1 = 0)."""
    rng = np.random.default_rng(seed)
    x1 = rng.uniform(-150e-6, 150e-6, n)
    u1 = _field(rng, n)
    w = np.full(n, 9e-6)
    g = dict(m2=18, p2=13e-6, lam=lam, z0=z0, s=s)
    r0 = z0 - c
    k = 2 * np.pi / lam
    sz = np.sqrt(1 - s ** 2)
    ref = line(dict(g, z0=r0), x1, np.zeros(n), w, u1, 7) * np.sqrt(r0 / z0) * np.exp(1j * k * sz * c)
    return rel_l2(line(g, x1, np.full(n, c), w, u1, 5), ref)


def pin_eq2_depth_shift(line, c=0.3e-3, n=32, lam=633e-9, z0=0.05, s=-0.015, seed=45):
    """d1 = c: Eq. 2 equals z0/(z0 - c) exp(ik sz c) times Eq. 2 of the flat
    source at distance z0 - c."""
    rng = np.random.default_rng(seed)
    x1 = rng.uniform(-150e-6, 150e-6, n)
    u1 = _field(rng, n)
    w = np.full(n, 9e-6)
    g = dict(m2=16, p2=15e-6, lam=lam, z0=z0, s=s)
    k = 2 * np.pi / lam
    sz = np.sqrt(1 - s ** 2)
    ref = line(dict(g, z0=z0 - c), x1, np.zeros(n), w, u1, 2) * (z0 / (z0 - c)) * np.exp(1j * k * sz * c)
    return rel_l2(line(g, x1, np.full(n, c), w, u1, 2), ref)


def pin_eq2_fresnel_limit(line, n=32, p1=20e-6, lam=633e-9, seed=46):
    """Eq. 2 -> Eq. 5 as the distance grows, for a flat source: the amplitude
    z0 r^-3/2 = z0^-1/2 (1 + dx^2/z0^2)^-3/4 and the Fresnel phase k dx^4/(8 z0^3)
    differ by terms of order 1/z0^2, so doubling z0 cuts the difference at
    least threefold, and at 1 m over this 0.6 mm aperture it is below 1e-6.
    Returns the largest measurement over its bound (pass: < 1)."""
    rng = np.random.default_rng(seed)
    x1 = _uniform(n, p1)
    u1 = _field(rng, n)
    w = np.full(n, p1)
    d1 = np.zeros(n)
    errs = []
    for z0 in (0.25, 0.5, 1.0):
        g = dict(m2=12, p2=25e-6, lam=lam, z0=z0)
        errs.append(rel_l2(line(g, x1, d1, w, u1, 2), line(g, x1, d1, w, u1, 5)))
    return max(errs[1] / errs[0] * 3, errs[2] / errs[1] * 3, errs[2] / 1e-6)


LINE_PINS = {
    "fft_natural_pitch": (pin_fft_natural_pitch, 1e-9),
    "planar_shift": (pin_planar_shift, 1e-9),
    "gaussian": (pin_gaussian, 1e-9),
    "permute_and_split": (pin_permute_and_split, 1e-12),
    "eq5_equals_eq7_flat": (pin_eq5_equals_eq7_flat, 1e-9),
    "eq5_planar_shift": (pin_eq5_planar_shift, 1e-9),
    "eq2_depth_shift": (pin_eq2_depth_shift, 1e-9),
    "eq2_fresnel_limit": (pin_eq2_fresnel_limit, 1.0),
}
