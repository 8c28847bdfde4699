"""Seeded synthetic workloads (source surfaces and fields).

This module only generates inputs: height maps d1 and complex source fields
u1 on the uniform source grid, with the shapes, sizes and value distributions
of the five standard workloads.  It holds none of the diffraction arithmetic
and is shared, read-only, by the CUDA path's tests, the benchmark and the
oracle's tests.

Coordinates follow the library's convention x1 = ((n - N/2) p), so the grid is
centred on the optical axis.  All arrays are row-major [y][x].  u1 is returned
as complex64 (the precision the CUDA path consumes) so that every consumer sees
bit-identical field values; d1 is float64 metres.
"""
from __future__ import annotations

import math

import numpy as np

NM = 1e-9
UM = 1e-6
MM = 1e-3


def geometry(n1x, n1y, p1x, p1y, m2x, m2y, p2x, p2y, lam, z0):
    """Plain dict of the grid geometry used by every consumer (SI units)."""
    return dict(n1x=int(n1x), n1y=int(n1y), p1x=float(p1x), p1y=float(p1y),
                m2x=int(m2x), m2y=int(m2y), p2x=float(p2x), p2y=float(p2y),
                lam=float(lam), z0=float(z0))


def coords(n: int, p: float) -> np.ndarray:
    """Centred sample coordinates (n - N/2) p."""
    return (np.arange(n) - n // 2) * p


# --- surfaces --------------------------------------------------------------

def surface_sinusoid(g, amp, period):
    """d1 = amp sin(2 pi x / period) sin(2 pi y / period)."""
    x = coords(g["n1x"], g["p1x"])
    y = coords(g["n1y"], g["p1y"])
    return amp * np.sin(2 * np.pi * y / period)[:, None] * np.sin(2 * np.pi * x / period)[None, :]


def surface_spherical_cap(g, radius):
    """Spherical cap sqrt(R^2 - rho^2) - sqrt(R^2 - rho_max^2), rho_max = half-diagonal."""
    x = coords(g["n1x"], g["p1x"])
    y = coords(g["n1y"], g["p1y"])
    rho2 = y[:, None] ** 2 + x[None, :] ** 2
    rho_max2 = (g["n1x"] / 2 * g["p1x"]) ** 2 + (g["n1y"] / 2 * g["p1y"]) ** 2
    return np.sqrt(radius ** 2 - rho2) - np.sqrt(radius ** 2 - rho_max2)


def surface_smooth_random(g, rng, sigma_samples, pv):
    """Gaussian noise smoothed by a periodic Gaussian filter of std sigma_samples,
    rescaled affinely to [0, pv]."""
    noise = rng.standard_normal((g["n1y"], g["n1x"]))
    fy = np.fft.fftfreq(g["n1y"])[:, None]
    fx = np.fft.fftfreq(g["n1x"])[None, :]
    transfer = np.exp(-2 * np.pi ** 2 * sigma_samples ** 2 * (fx ** 2 + fy ** 2))
    s = np.fft.ifft2(np.fft.fft2(noise) * transfer).real
    s -= s.min()
    return s * (pv / s.max())


def surface_tilt_bump(g, tilt_deg, bump_height, bump_sigma):
    """Plane tilted about the y axis through the centre plus a centred Gaussian bump."""
    x = coords(g["n1x"], g["p1x"])
    y = coords(g["n1y"], g["p1y"])
    tilt = np.broadcast_to(x[None, :] * math.tan(math.radians(tilt_deg)), (g["n1y"], g["n1x"]))
    rho2 = y[:, None] ** 2 + x[None, :] ** 2
    return tilt + bump_height * np.exp(-rho2 / (2 * bump_sigma ** 2))


# --- fields ------------------------------------------------------------------

def field_unit(g):
    return np.ones((g["n1y"], g["n1x"]), np.complex64)


def field_binary_mask(g, rng, p=0.5):
    return (rng.random((g["n1y"], g["n1x"])) < p).astype(np.complex64)


def field_random_amp_phase(g, rng):
    amp = rng.random((g["n1y"], g["n1x"]))
    ph = rng.random((g["n1y"], g["n1x"])) * 2 * np.pi
    return (amp * np.exp(1j * ph)).astype(np.complex64)


def field_unit_random_phase(g, rng):
    ph = rng.random((g["n1y"], g["n1x"])) * 2 * np.pi
    return np.exp(1j * ph).astype(np.complex64)


# --- the standard workloads ---------------------------------------------------

WORKLOADS = ("sinusoid64", "spherical_cap1024", "smooth_random2048", "rgb_batch24", "tilt_bump4096")


def make(name: str, seed: int | None = None, scale: int = 1):
    """Return (geometry, u1 complex64 [n1y, n1x], d1 float64 [n1y, n1x]).

    name is one of WORKLOADS except the batch (see make_batch).  scale > 1
    divides the grid sizes by scale while keeping pitch, wavelength and
    distance (a smaller case of the same workload, for quick parity runs).
    """
    if name == "sinusoid64":
        n = 64 // scale
        g = geometry(n, n, 10 * UM, 10 * UM, n, n, 10 * UM, 10 * UM, 633 * NM, 0.05)
        return g, field_unit(g), surface_sinusoid(g, 20 * UM, 320 * UM)
    if name == "spherical_cap1024":
        rng = np.random.default_rng(2 if seed is None else seed)
        n = 1024 // scale
        g = geometry(n, n, 8 * UM, 8 * UM, n, n, 8 * UM, 8 * UM, 532 * NM, 0.2)
        return g, field_binary_mask(g, rng), surface_spherical_cap(g, 20 * MM)
    if name == "smooth_random2048":
        rng = np.random.default_rng(3 if seed is None else seed)
        n = 2048 // scale
        g = geometry(n, n, 4 * UM, 4 * UM, n, n, 4 * UM, 4 * UM, 633 * NM, 0.1)
        d1 = surface_smooth_random(g, rng, 40.0 / scale, 50 * UM)
        return g, field_random_amp_phase(g, rng), d1
    if name == "tilt_bump4096":
        rng = np.random.default_rng(5 if seed is None else seed)
        n = 4096 // scale
        p = 3.74 * UM
        g = geometry(n, n, p, p, n, n, p, p, 532 * NM, 0.15)
        return g, field_unit_random_phase(g, rng), surface_tilt_bump(g, 2.0, 30 * UM, 2 * MM)
    raise ValueError(f"unknown workload {name!r}")


def make_batch(seed: int = 4, count: int = 24, sizes=(256, 512, 1024, 2048), pitch=3 * UM):
    """The RGB batch: count surfaces of sizes drawn from `sizes`, wavelengths
    cycled over 450/532/633 nm, z0 ~ U[0.05, 0.3] m, sinusoidal or smooth
    random d1 with amplitude ~ U[5, 50] um, field with uniform amplitude and
    phase.  Returns a list of (geometry, u1, d1)."""
    rng = np.random.default_rng(seed)
    lams = (450 * NM, 532 * NM, 633 * NM)
    out = []
    for i in range(count):
        n = int(rng.choice(sizes))
        lam = lams[i % 3]
        z0 = float(rng.uniform(0.05, 0.3))
        amp = float(rng.uniform(5 * UM, 50 * UM))
        g = geometry(n, n, pitch, pitch, n, n, pitch, pitch, lam, z0)
        if rng.random() < 0.5:
            d1 = surface_sinusoid(g, amp, 320 * UM)
        else:
            d1 = surface_smooth_random(g, rng, 40.0, amp)
        out.append((g, field_random_amp_phase(g, rng), d1))
    return out


def sample_points(g, count: int, seed: int):
    """`count` distinct destination grid indices drawn without replacement.
    Returns (mx, my) int32 arrays."""
    rng = np.random.default_rng(seed)
    total = g["m2x"] * g["m2y"]
    flat = rng.choice(total, size=min(count, total), replace=False)
    return (flat % g["m2x"]).astype(np.int32), (flat // g["m2x"]).astype(np.int32)


# --- one-dimensional line sources (explicit samples along the surface) ------------

def line_geometry(m2: int = 1024, p2: float = 10 * UM, lam: float = 633e-9, z0: float = 1.0,
                  s: float = 0.0) -> dict:
    """Destination line and light of the paper's 1D experiments (Sec. 3):
    1024 destination points at 10 um, 633 nm, z0 = 1 m, normal incidence."""
    return dict(m2=m2, p2=p2, lam=lam, z0=z0, s=s)


def line_facets(n_facet: int = 128, p: float = 10 * UM,
                angles=(-30.0, -50.0, 0.0, 50.0)):
    """Tilted planar facets sampled every p along the surface (Sec. 3, first
    experiment).  Reading of the layout, which the paper does not give: four
    facets of n_facet samples at the given angles to x1, each preceded by a
    flat segment of n_facet samples (1024 samples in all), heights continuous,
    the line centred on x1 = 0.  Returns (x1, d1, w) with the projected weight
    w = p |cos(angle)| of each sample."""
    steps = []
    for a in angles:
        steps += [0.0] * n_facet + [float(a)] * n_facet
    ang = np.deg2rad(np.array(steps))
    dx = p * np.cos(ang)
    dz = p * np.sin(ang)
    x1 = np.cumsum(dx) - 0.5 * dx
    d1 = np.cumsum(dz) - 0.5 * dz
    x1 -= 0.5 * (x1[0] + x1[-1])
    d1 -= d1.mean()
    return x1, d1, np.abs(dx)


def line_quadratic(n: int = 1024, p: float = 10 * UM, max_slope: float = 1.0):
    """Quadratic curve d1 = a x1^2 sampled every p along its arc length (Sec. 3,
    second experiment).  Reading: the paper gives no coefficient; a is chosen so
    that the slope at the ends of the n samples is max_slope (45 degrees).
    Returns (x1, d1, w) with w = dx1 of each sample."""
    half = 0.5 * n * p

    def arclen(x, a):  # closed form of int_0^x sqrt(1 + (2 a t)^2) dt
        u = 2 * a * x
        return (u * np.sqrt(1 + u * u) + np.arcsinh(u)) / (4 * a)

    # the end x_e satisfies 2 a x_e = max_slope and arclen(x_e, a) = half
    m = max_slope
    a = (m * np.sqrt(1 + m * m) + np.arcsinh(m)) / (4 * half)
    s_mid = (np.arange(n) - n / 2 + 0.5) * p
    # invert the (odd, monotone) arc length by bisection on |s|
    target = np.abs(s_mid)
    lo, hi = np.zeros(n), np.full(n, 2 * half)
    for _ in range(80):
        mid = 0.5 * (lo + hi)
        big = arclen(mid, a) > target
        hi = np.where(big, mid, hi)
        lo = np.where(big, lo, mid)
    x1 = np.sign(s_mid) * 0.5 * (lo + hi)
    d1 = a * x1 ** 2
    d1 -= d1.mean()
    w = p / np.sqrt(1 + (2 * a * x1) ** 2)
    return x1, d1, w


def make_multi(seed: int = 6):
    """Several surfaces summed at one destination (a small CGH-like object):
    three source grids of 384^2, 256^2 and 512^2 samples at 8 um, placed at
    different positions (offsets), with a spherical cap, a sinusoid and a
    smooth random surface, random-phase fields; destination 1024^2 at 8 um,
    532 nm, z0 0.2 m.  Returns a list of (geometry, u1, d1)."""
    rng = np.random.default_rng(seed)
    items = []
    spec = [(384, (-1.2e-3, 0.6e-3), "cap"), (256, (1.0e-3, 1.1e-3), "sin"),
            (512, (0.2e-3, -0.9e-3), "smooth")]
    for n, (ox, oy), kind in spec:
        g = geometry(n, n, 8 * UM, 8 * UM, 1024, 1024, 8 * UM, 8 * UM, 532e-9, 0.2)
        g = dict(g, ox=ox, oy=oy)
        if kind == "cap":
            d1 = surface_spherical_cap(g, 15e-3)
        elif kind == "sin":
            d1 = surface_sinusoid(g, 15e-6, 400e-6)
        else:
            d1 = surface_smooth_random(g, rng, 30.0, 40e-6)
        items.append((g, field_random_amp_phase(g, rng), d1))
    return items
