"""Pins for the FP64 oracle: references that do not reuse the oracle's formula.

Each pin takes an ``eq7(g, u1, d1, points=None)`` callable (the oracle, or a
deliberately broken copy of it in the mutation test) and returns the relative
L2 error against a reference computed by another route:

* ``pin_fft_natural_pitch`` -- d1 = 0 at the natural destination pitch
  p2 = lambda z0 / (N p1): the sum is a centred 2D DFT, computed with numpy's
  FFT (Sec. 2, Eq. 7 with d1 = 0 reduces to single-FFT Fresnel diffraction).
* ``pin_planar_shift`` -- d1 = c: Eq. 7 equals single-FFT planar Fresnel
  propagation over z0 - c (numpy FFT at that distance's natural pitch), times
  exp(ik c) times the two factors the approximations of Eqs. 5-6 leave:
  (z0 - c)/z0 and exp(ik|x2|^2 (1/z0 - 1/(z0 - c))/2).
* ``pin_gaussian`` -- a Gaussian source on d1 = c: the continuous integral
  has a closed form; the discrete sum matches it to truncation and aliasing
  error (chosen below 1e-9).
* ``pin_terraces`` -- piecewise-constant d1: by linearity the result is a
  sum over terraces of separable transforms, each computed as two dense 1D
  DFT matrix products per axis (exercises a per-sample r0 and the x/y roles
  with non-square grids and unequal pitches).
* ``pin_single_sample_modulus`` -- one nonzero sample: |u2| = p1x p1y |u1| /
  (lambda z0) at every destination point.
"""
from __future__ import annotations

import numpy as np


def _coords(n, p):
    return (np.arange(n) - n // 2) * p


def rel_l2(a, b):
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def centred_dft2(f):
    """F[m'] = sum_n f[n] exp(-2 pi i n' m'/N) with centred indices (library FFT)."""
    return np.fft.fftshift(np.fft.fft2(np.fft.ifftshift(f)))


def planar_fresnel_fft(u1, p1x, p1y, lam, z):
    """Textbook single-FFT Fresnel propagation over distance z (Goodman, Ch. 4):
    U(x2) = e^{ikz} e^{ik|x2|^2/2z} / (i lam z) * FT[u1 e^{ik|x1|^2/2z}] at
    the natural pitch p2 = lam z / (N p1).  Returns (U, p2x, p2y)."""
    n1y, n1x = u1.shape
    k = 2 * np.pi / lam
    x = _coords(n1x, p1x)[None, :]
    y = _coords(n1y, p1y)[:, None]
    p2x = lam * z / (n1x * p1x)
    p2y = lam * z / (n1y * p1y)
    X = _coords(n1x, p2x)[None, :]
    Y = _coords(n1y, p2y)[:, None]
    F = centred_dft2(u1 * np.exp(1j * k * (x ** 2 + y ** 2) / (2 * z))) * p1x * p1y
    U = np.exp(1j * k * z) * np.exp(1j * k * (X ** 2 + Y ** 2) / (2 * z)) / (1j * lam * z) * F
    return U, p2x, p2y


def _rng_field(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def pin_fft_natural_pitch(eq7, n1x=24, n1y=16, p1x=10e-6, p1y=7e-6, lam=633e-9, z0=0.05, seed=11):
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    U, p2x, p2y = planar_fresnel_fft(u1, p1x, p1y, lam, z0)
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=n1x, m2y=n1y, p2x=p2x, p2y=p2y,
             lam=lam, z0=z0)
    return rel_l2(eq7(g, u1, np.zeros((n1y, n1x))), U)


def pin_planar_shift(eq7, c=0.3e-3, n1x=20, n1y=16, p1x=10e-6, p1y=8e-6, lam=633e-9, z0=0.05,
                     seed=12):
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    z = z0 - c
    U, p2x, p2y = planar_fresnel_fft(u1, p1x, p1y, lam, z)
    k = 2 * np.pi / lam
    X = _coords(n1x, p2x)[None, :]
    Y = _coords(n1y, p2y)[:, None]
    ref = U * np.exp(1j * k * c) * (z / z0) * np.exp(
        1j * k * (X ** 2 + Y ** 2) * (1 / z0 - 1 / z) / 2)
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=n1x, m2y=n1y, p2x=p2x, p2y=p2y,
             lam=lam, z0=z0)
    return rel_l2(eq7(g, u1, np.full((n1y, n1x), c)), ref)


def pin_gaussian(eq7, c=0.2e-3, n1=64, p1=10e-6, m2x=40, m2y=36, p2x=11e-6, p2y=13e-6,
                 lam=633e-9, z0=0.05):
    """Gaussian u1 = exp(-|x1|^2/w0^2) on the plane d1 = c (w0 = aperture/10).
    With r0 = z0 - c and a = 1/w0^2 - ik/(2 r0), the integral over x1 of
    u1 e^{ik|x1|^2/2r0} e^{-ik x1.x2/r0} is (pi/a) exp(-(k/r0)^2 |x2|^2/(4a))."""
    k = 2 * np.pi / lam
    w0 = n1 * p1 / 10
    x = _coords(n1, p1)
    u1 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / w0 ** 2).astype(np.complex128)
    r0 = z0 - c
    a = 1 / w0 ** 2 - 1j * k / (2 * r0)
    X = _coords(m2x, p2x)[None, :]
    Y = _coords(m2y, p2y)[:, None]
    r2 = X ** 2 + Y ** 2
    integral = (np.pi / a) * np.exp(-(k / r0) ** 2 * r2 / (4 * a))
    ref = np.exp(1j * k * (z0 + r2 / (2 * z0))) / (1j * lam * z0) * integral
    g = dict(n1x=n1, n1y=n1, p1x=p1, p1y=p1, m2x=m2x, m2y=m2y, p2x=p2x, p2y=p2y, lam=lam, z0=z0)
    return rel_l2(eq7(g, u1, np.full((n1, n1), c)), ref)


def pin_gaussian_tilted(eq7, c=0.15e-3, sx=0.0021, sy=-0.0013, n1=64, p1=10e-6, m2x=40, m2y=36,
                        p2x=11e-6, p2y=13e-6, lam=633e-9, z0=0.05):
    """The Gaussian of pin_gaussian lit by a plane wave with direction cosines
    (sx, sy): u_I = exp(ik(s.x1 + sz c)) on the plane d1 = c.  The linear phase
    moves the Gaussian integral to x2 - r0 s and the depth term leaves the
    constant exp(ik c (sz - 1)) next to the exp(-ik c) of Eq. 5.  The tilt
    keeps the moved beam inside the destination window (r0 |s| ~ 0.1 mm)."""
    k = 2 * np.pi / lam
    w0 = n1 * p1 / 10
    x = _coords(n1, p1)
    u1 = np.exp(-(x[None, :] ** 2 + x[:, None] ** 2) / w0 ** 2).astype(np.complex128)
    r0 = z0 - c
    sz = np.sqrt(1 - sx ** 2 - sy ** 2)
    a = 1 / w0 ** 2 - 1j * k / (2 * r0)
    X = _coords(m2x, p2x)[None, :]
    Y = _coords(m2y, p2y)[:, None]
    r2s = (X - r0 * sx) ** 2 + (Y - r0 * sy) ** 2
    integral = (np.pi / a) * np.exp(-(k / r0) ** 2 * r2s / (4 * a))
    ref = (np.exp(1j * k * (z0 + (X ** 2 + Y ** 2) / (2 * z0))) / (1j * lam * z0)
           * np.exp(1j * k * c * (sz - 1)) * integral)
    g = dict(n1x=n1, n1y=n1, p1x=p1, p1y=p1, m2x=m2x, m2y=m2y, p2x=p2x, p2y=p2y, lam=lam, z0=z0,
             sx=sx, sy=sy)
    return rel_l2(eq7(g, u1, np.full((n1, n1), c)), ref)


def pin_terraces(eq7, n1x=18, n1y=14, p1x=9e-6, p1y=6e-6, m2x=12, m2y=22, p2x=15e-6, p2y=5e-6,
                 lam=532e-9, z0=0.04, seed=13):
    """d1 takes four constant values on random masks.  For one terrace with
    height c and r0 = z0 - c the sum factorises per axis:
      S_c = Ey (M_c o u1 o Cy Cx^T) Ex^T,  Ex[m, n] = exp(-ik x1[n] x2[m] / r0),
    with the source chirp split as Cy[ny] Cx[nx] = exp(ik(x^2 + y^2)/(2 r0))."""
    rng = np.random.default_rng(seed)
    k = 2 * np.pi / lam
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    heights = np.array([-0.4e-3, 0.0, 0.25e-3, 0.9e-3])
    label = rng.integers(0, heights.size, (n1y, n1x))
    d1 = heights[label]
    x1 = _coords(n1x, p1x)
    y1 = _coords(n1y, p1y)
    x2 = _coords(m2x, p2x)
    y2 = _coords(m2y, p2y)
    total = np.zeros((m2y, m2x), np.complex128)
    for t, c in enumerate(heights):
        r0 = z0 - c
        Ex = np.exp(-1j * k * np.outer(x2, x1) / r0)          # [m2x, n1x]
        Ey = np.exp(-1j * k * np.outer(y2, y1) / r0)          # [m2y, n1y]
        chirp = np.outer(np.exp(1j * k * y1 ** 2 / (2 * r0)), np.exp(1j * k * x1 ** 2 / (2 * r0)))
        f = np.where(label == t, u1 * chirp, 0)
        total += Ey @ f @ Ex.T
    X, Y = x2[None, :], y2[:, None]
    outer = np.exp(1j * k * (z0 + (X ** 2 + Y ** 2) / (2 * z0))) / (1j * lam * z0)
    ref = outer * p1x * p1y * total
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=m2x, m2y=m2y, p2x=p2x, p2y=p2y,
             lam=lam, z0=z0)
    return rel_l2(eq7(g, u1, d1), ref)


def pin_single_sample_modulus(eq7, n1=16, p1=10e-6, lam=633e-9, z0=0.05, seed=14):
    rng = np.random.default_rng(seed)
    u1 = np.zeros((n1, n1), np.complex128)
    a = 0.7 - 0.3j
    u1[3, 11] = a
    d1 = rng.uniform(-50e-6, 50e-6, (n1, n1))
    g = dict(n1x=n1, n1y=n1, p1x=p1, p1y=p1, m2x=n1, m2y=n1, p2x=12e-6, p2y=9e-6, lam=lam, z0=z0)
    out = eq7(g, u1, d1)
    expect = p1 * p1 * abs(a) / (lam * z0)
    return float(np.max(np.abs(np.abs(out) - expect)) / expect)


def pin_offset_is_padding(eq7, n1x=12, n1y=10, sx_=3, sy_=-2, p1x=10e-6, p1y=8e-6, lam=633e-9,
                          z0=0.05, seed=15):
    """A source grid placed off the axis by whole samples, (ox, oy) =
    (3 p1x, -2 p1y), equals the same samples embedded at shifted indices in a
    larger zero-padded grid centred on the axis (zero samples add nothing)."""
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    d1 = rng.uniform(-40e-6, 40e-6, (n1y, n1x))
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=14, m2y=12, p2x=12e-6, p2y=11e-6,
             lam=lam, z0=z0, ox=sx_ * p1x, oy=sy_ * p1y)
    big_x, big_y = n1x + 2 * abs(sx_) + 2, n1y + 2 * abs(sy_) + 2
    ub = np.zeros((big_y, big_x), np.complex128)
    db = np.zeros((big_y, big_x))
    x0 = big_x // 2 - n1x // 2 + sx_
    y0 = big_y // 2 - n1y // 2 + sy_
    ub[y0:y0 + n1y, x0:x0 + n1x] = u1
    db[y0:y0 + n1y, x0:x0 + n1x] = d1
    gb = dict(g, n1x=big_x, n1y=big_y, ox=0.0, oy=0.0)
    return rel_l2(eq7(g, u1, d1), eq7(gb, ub, db))


# Tolerances: the phases k z0 ~ 5e5 rad carry FP64 rounding of ~1e-10 rad, so
# agreement is bounded near 1e-10; every planted mistake gives O(1) errors.
ALL_PINS = {
    "fft_natural_pitch": (pin_fft_natural_pitch, 1e-9),
    "planar_shift": (pin_planar_shift, 1e-9),
    "gaussian": (pin_gaussian, 1e-9),
    "gaussian_tilted": (pin_gaussian_tilted, 1e-9),
    "terraces": (pin_terraces, 1e-9),
    "single_sample_modulus": (pin_single_sample_modulus, 1e-12),
    "offset_is_padding": (pin_offset_is_padding, 1e-12),
}


# --- Eq. 5 and Eq. 2 (direct sums before the approximations of Eqs. 4 and 6) ---------

def pin_eq5_equals_eq7_flat(eq5, eq2, eq7, n1x=20, n1y=14, p1x=10e-6, p1y=8e-6, lam=633e-9,
                            z0=0.05, seed=31):
    """d1 = 0: r0 = z0 everywhere, so Eq. 6 is exact and Eq. 5 is Eq. 7."""
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=16, m2y=18, p2x=12e-6, p2y=9e-6,
             lam=lam, z0=z0)
    d1 = np.zeros((n1y, n1x))
    return rel_l2(eq5(g, u1, d1), eq7(g, u1, d1))


def pin_eq5_planar_shift(eq5, eq2, eq7, c=0.4e-3, n1x=18, n1y=16, p1x=10e-6, p1y=7e-6,
                         lam=532e-9, z0=0.04, sx=0.017, sy=0.011, seed=32):
    """d1 = c under a plane wave with direction cosines (sx, sy): the
    exponentials of Eq. 5 combine to exp(ik s.x1) exp(ik c (sz - 1))
    exp(ik|x1 - x2|^2/(2 (z0 - c))), i.e. planar Fresnel propagation of the lit
    field over z0 - c with the prefactor exp(ik z0)/(i lambda z0) instead of
    exp(ik(z0 - c))/(i lambda (z0 - c)); that propagation is Eq. 7 at d1 = 0."""
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=14, m2y=20, p2x=11e-6, p2y=13e-6,
             lam=lam, z0=z0, sx=sx, sy=sy)
    r0 = z0 - c
    gz = dict(g, z0=r0)
    k = 2 * np.pi / lam
    sz = np.sqrt(1 - sx ** 2 - sy ** 2)
    ref = eq7(gz, u1, np.zeros((n1y, n1x))) * (r0 / z0) * np.exp(1j * k * c * sz)
    return rel_l2(eq5(g, u1, np.full((n1y, n1x), c)), ref)


def pin_eq2_depth_shift(eq5, eq2, eq7, c=0.3e-3, n1x=16, n1y=14, p1x=10e-6, p1y=9e-6,
                        lam=633e-9, z0=0.05, sx=-0.012, sy=0.02, seed=33):
    """d1 = c: Eq. 2 depends on the surface height only through u_I =
    exp(ik(s.x1 + sz c)) and the distance z0 - c, so it equals
    z0/(z0 - c) exp(ik sz c) times Eq. 2 of the flat surface at distance z0 - c."""
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1y, n1x)).astype(np.complex128)
    g = dict(n1x=n1x, n1y=n1y, p1x=p1x, p1y=p1y, m2x=12, m2y=10, p2x=15e-6, p2y=14e-6,
             lam=lam, z0=z0, sx=sx, sy=sy)
    k = 2 * np.pi / lam
    sz = np.sqrt(1 - sx ** 2 - sy ** 2)
    ref = (eq2(dict(g, z0=z0 - c), u1, np.zeros((n1y, n1x))) * (z0 / (z0 - c))
           * np.exp(1j * k * c * sz))
    return rel_l2(eq2(g, u1, np.full((n1y, n1x), c)), ref)


def pin_eq2_fresnel_limit(eq5, eq2, eq7, n1=16, p1=20e-6, lam=633e-9, seed=34):
    """Eq. 2 -> Eq. 5 as the distance grows: the largest neglected term is the
    amplitude of r^2 ~ z0^2, a relative 2 d1/z0 for a surface of height d1
    (here +-20 um), then the Fresnel expansion's (Eq. 4) 1/z0^2 and 1/z0^3
    terms, so doubling z0 must cut the difference at least 1.8-fold, and at
    z0 = 1 m over this 0.3 mm aperture it is below 1e-5.  Returns the largest of
    the three measurements over its bound (pass: < 1)."""
    rng = np.random.default_rng(seed)
    u1 = _rng_field(rng, (n1, n1)).astype(np.complex128)
    d1 = rng.uniform(-20e-6, 20e-6, (n1, n1))
    errs = []
    for z0 in (0.25, 0.5, 1.0):
        g = dict(n1x=n1, n1y=n1, p1x=p1, p1y=p1, m2x=12, m2y=12, p2x=25e-6, p2y=25e-6,
                 lam=lam, z0=z0)
        errs.append(rel_l2(eq2(g, u1, d1), eq5(g, u1, d1)))
    return max(errs[1] / errs[0] * 1.8, errs[2] / errs[1] * 1.8, errs[2] / 1e-5)


DIRECT_PINS = {
    "eq5_equals_eq7_flat": (pin_eq5_equals_eq7_flat, 1e-9),
    "eq5_planar_shift": (pin_eq5_planar_shift, 1e-9),
    "eq2_depth_shift": (pin_eq2_depth_shift, 1e-9),
    "eq2_fresnel_limit": (pin_eq2_fresnel_limit, 1.0),
}
