"""Smallest error any width-w gridding can reach in the NUFFT of Eq. 8.

TEST INFRASTRUCTURE ONLY (same rule as the rest of ``oracle/``): only
``tests/`` may import this module.  Plain numpy/scipy in FP64; it shares no
code with the CUDA library.

Sec. 2 (after Eq. 9) evaluates the Fourier form of Eq. 7 with a type-1 NUFFT:
each sample value c_j is spread onto an oversampled grid (sigma M cells per
axis) around its non-uniform coordinate g_j, the grid is Fourier transformed,
and the M kept modes are divided by the kernel's transform.  Only the
gridding kernel differs between the exponential-of-semicircle kernel, the
Gaussian of Greengard and Lee, and a learned tabulated kernel.  This module
asks what the best possible width-w gridding achieves.

Model (one axis; ``delta`` = sub-cell offset of a sample, tap i at distance
o_i(delta) = delta - w/2 + i from it, i = 0..w-1; omega = 2 pi m / (sigma M),
|omega| <= pi/sigma for the kept modes m):
  the gridded-and-transformed sample contributes to mode m
      R(omega, delta) = sum_i W_i(delta) exp(-i omega o_i(delta))
  times its exact term exp(-i omega g_j); after a per-mode correction H(omega)
  the relative error of that contribution is H R - 1.
For sample values that are independent with zero mean (random phase, as in
the 2048^2 smooth-random workload) the errors of different samples add in
energy, so the expected squared relative L2 error over the kept modes is
      E1 = mean over delta and omega of |H(omega) R(omega, delta) - 1|^2
with delta uniform on [0, 1) (the offsets of a non-integer lattice spacing
are equidistributed).  Any tap table W(delta) -- one weight function per tap,
of any shape, per tile or global -- and any correction H are covered.  For
fixed H the best W(delta) is a least-squares solution per delta; what is
left is a function of H alone (variable projection), minimised here by
L-BFGS over log H.  In 2D with the product kernel W_x(dx) W_y(dy) and
H_x H_y, the error is 1 - (1 - E1)^2 at the optimal overall scale (see
``floor_2d_from_1d``), and ``nonseparable_floor_2d`` checks that a full
w x w table per (dx, dy) with a non-separable H reaches no lower.
"""
from __future__ import annotations

import numpy as np
from scipy.optimize import minimize


def es_weights(z: np.ndarray, w: int, beta: float) -> np.ndarray:
    """Exponential-of-semicircle kernel exp(beta (sqrt(1 - (2z/w)^2) - 1)) on |z| < w/2."""
    u = 2.0 * np.asarray(z, np.float64) / w
    out = np.zeros_like(u)
    m = np.abs(u) < 1.0
    out[m] = np.exp(beta * (np.sqrt(1.0 - u[m] ** 2) - 1.0))
    return out


def tap_offsets(delta: np.ndarray, w: int) -> np.ndarray:
    """o_i(delta) = delta - w/2 + i: distance of tap i from the sample
    (delta in [0, 1) is the offset of the first tap, w/2 - delta cells below)."""
    return np.asarray(delta, np.float64)[:, None] - 0.5 * w + np.arange(w)[None, :]


def grids(w: int, sigma: float, nd: int, nw: int, omega: np.ndarray | None = None):
    """Midpoint grids of delta on [0, 1) and omega on [-pi/sigma, pi/sigma)
    (or the given omega), and A[d, o, i] = exp(-i omega_o o_i(delta_d))."""
    delta = (np.arange(nd) + 0.5) / nd
    if omega is None:
        omega = ((np.arange(nw) + 0.5) / nw * 2.0 - 1.0) * np.pi / sigma
    omega = np.asarray(omega, np.float64)
    A = np.exp(-1j * omega[None, :, None] * tap_offsets(delta, w)[:, None, :])
    return delta, omega, A


def mode_omegas(M: int, sigma: float = 2.0) -> np.ndarray:
    """omega = 2 pi m / (sigma M) of the kept modes m in [-M/2, M/2)."""
    return 2.0 * np.pi * np.arange(-M // 2, M // 2) / (sigma * M)


def error_of(W: np.ndarray, H: np.ndarray, A: np.ndarray) -> float:
    """E1 for tap weights W[d, i] and correction H[o]."""
    R = np.einsum("doi,di->do", A, W)
    return float(np.mean(np.abs(H[None, :] * R - 1.0) ** 2))


def best_correction(W: np.ndarray, A: np.ndarray) -> np.ndarray:
    """H minimising E1 for fixed W: H = mean_d conj(R) / mean_d |R|^2 per omega."""
    R = np.einsum("doi,di->do", A, W)
    return np.mean(np.conj(R), axis=0) / np.mean(np.abs(R) ** 2, axis=0)


def best_weights(H: np.ndarray, A: np.ndarray) -> np.ndarray:
    """Least-squares W(delta) for fixed real H: min_W sum_o |H_o (A W)_o - 1|^2."""
    M = A * H[None, :, None]
    G = np.einsum("doi,doj->dij", np.conj(M), M)
    r = np.einsum("doi->di", np.conj(M))
    return np.linalg.solve(G, r[..., None])[..., 0]


def _varpro(logh: np.ndarray, A: np.ndarray):
    """E1 with W eliminated, and its gradient with respect to log H (H real, > 0).

    proj_d = r^H G^-1 r with r = A^H H, G = A^H diag(H^2) A; E1 = mean_d (1 - proj_d / n).
    d proj_d / d H_o = 2 Re (A x)_o - 2 H_o |(A x)_o|^2 with x = G^-1 r."""
    H = np.exp(logh)
    n = A.shape[1]
    M = A * H[None, :, None]
    G = np.einsum("doi,doj->dij", np.conj(M), M)
    r = np.einsum("doi,o->di", np.conj(A), H)
    x = np.linalg.solve(G, r[..., None])[..., 0]
    proj = np.real(np.einsum("di,di->d", np.conj(r), x))
    Ax = np.einsum("doi,di->do", A, x)
    dproj = 2.0 * np.real(Ax) - 2.0 * H[None, :] * np.abs(Ax) ** 2
    e = float(np.mean(1.0 - proj / n))
    grad = -np.mean(dproj, axis=0) / n * H
    return e, grad


def floor_1d(w: int, sigma: float = 2.0, nd: int = 128, nw: int = 256, beta: float | None = None,
             h0: np.ndarray | None = None, omega: np.ndarray | None = None):
    """Minimum of E1 over every tap table and correction.  Returns
    (E1_min, H, W, delta, omega).  The search starts from the correction of the
    ES kernel (beta = 2.30 w unless given) or from h0."""
    delta, omega, A = grids(w, sigma, nd, nw, omega)
    if h0 is None:
        b = 2.30 * w if beta is None else beta
        h0 = np.real(best_correction(es_weights(tap_offsets(delta, w), w, b), A))
    res = minimize(_varpro, np.log(np.abs(h0)), args=(A,), jac=True, method="L-BFGS-B",
                   options={"maxiter": 5000, "ftol": 1e-16, "gtol": 1e-14, "maxcor": 30})
    H = np.exp(res.x)
    W = best_weights(H, A)
    return error_of(W, H, A), H, W, delta, omega


def es_error_1d(w: int, beta: float, sigma: float = 2.0, nd: int = 128, nw: int = 256,
                omega: np.ndarray | None = None) -> float:
    """E1 of the ES kernel with its best per-mode correction."""
    delta, omega, A = grids(w, sigma, nd, nw, omega)
    W = es_weights(tap_offsets(delta, w), w, beta)
    return error_of(W, best_correction(W, A), A)


def floor_2d_from_1d(e1: float) -> float:
    """Squared 2D relative error of the product of two identical 1D designs
    at their best common scale: 1 - (1 - E1)^2.

    With P = H R per axis, a = mean |P|^2 and b = mean P (over delta and
    omega), the 2D error is a_x a_y - 2 Re(b_x b_y) + 1; scaling P by c and
    minimising over c gives 1 - (b^2/a)^2 = 1 - (1 - E1)^2, since the 1D error
    at its own best scale is 1 - b^2/a."""
    return 1.0 - (1.0 - e1) ** 2


def nonseparable_floor_2d(w: int, sigma: float = 2.0, nd: int = 12, nw: int = 24,
                          h0: np.ndarray | None = None) -> float:
    """Squared 2D error minimised over a full w x w tap table per (dx, dy) and a
    non-separable correction H(omega_x, omega_y), on coarse grids."""
    _, _, A1 = grids(w, sigma, nd, nw)
    A = np.einsum("aoi,bpj->abopij", A1, A1).reshape(nd * nd, nw * nw, w * w)
    if h0 is None:
        h0 = np.ones(nw * nw)
    res = minimize(_varpro, np.log(h0), args=(A,), jac=True, method="L-BFGS-B",
                   options={"maxiter": 3000, "ftol": 1e-16, "gtol": 1e-14, "maxcor": 30})
    return float(res.fun)


def nufft_1d_direct_error(W_of_delta, H_of_omega, w: int, M: int = 256, sigma: float = 2.0,
                          n: int = 4000, seed: int = 0) -> float:
    """Relative L2 error of a brute-force 1D type-1 NUFFT against the direct
    sum, for independent random complex sample values at uniformly random
    positions: spread with W_of_delta(delta) (taps at first + i), FFT of the
    sigma M cells, keep modes m in [-M/2, M/2), multiply by H_of_omega.  An
    independent check of the error model above (explicit loops and numpy's
    FFT; nothing is shared with ``error_of``)."""
    rng = np.random.default_rng(seed)
    nf = int(round(sigma * M))
    g = rng.uniform(0.0, nf, n)                       # positions in cells
    c = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    grid = np.zeros(nf, np.complex128)
    for gj, cj in zip(g, c):
        first = int(np.ceil(gj - 0.5 * w))
        delta = first - (gj - 0.5 * w)               # in [0, 1)
        wt = W_of_delta(delta)
        for i in range(w):
            grid[(first + i) % nf] += cj * wt[i]
    m = np.arange(-M // 2, M // 2)
    F = np.array([np.sum(grid * np.exp(-2j * np.pi * mm * np.arange(nf) / nf)) for mm in m])
    omega = 2.0 * np.pi * m / nf
    approx = F * np.asarray(H_of_omega(omega))
    exact = np.array([np.sum(c * np.exp(-1j * om * g)) for om in omega])
    return float(np.linalg.norm(approx - exact) / np.linalg.norm(exact))
