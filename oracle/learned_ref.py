"""FP64 CPU reference of the learned-kernel forward map (test infrastructure).

TEST INFRASTRUCTURE ONLY, like the rest of oracle/: only tests/ may use it.

The learned kernel is an extension of the paper's method: Eq. 8 evaluated as
a type-1 NUFFT whose spreading kernel is a per-source-tile table predicted by
an MLP, with a learned deconvolution correction.  This module restates that
definition (the model layout documented in include/asfd.h) in plain numpy
FP64, with no shared code or tables with the CUDA library:

  sample n: c_n = u1[n] exp(ik d1) exp(ik(-d1 + |x1|^2/(2 r0)))     (Eq. 5, 8)
            G_n = p1 p2 nf/(lambda z0) x~ z0/r0 + nf/2 per axis     (fine grid)
            first tap l0 = ceil(G - 2), offset dx = l0 - (G - 2)
  tap a:    weight P_{tile, axis, a}(2 dx - 1), polynomial of degree 7
  grid:     b[l0 + a (mod nf)] += c_n P_x,a P_y,b
  u2[m]  =  exp(ik(z0 + |x2|^2/(2 z0))) / (i lambda z0) p1x p1y
            (-1)^(m'x + m'y) corr_x(m'x) corr_y(m'y) / (psi_x psi_y)
            sum_s b_s exp(-2 pi i m'.s / nf)
  psi = Fourier transform of the ES kernel of width 4 (beta = 9.2) at
  2 pi m'/nf (Gauss-Legendre quadrature), corr = 1 + sum_j d_j T_2j(2 m'/M).

Parity of this reference itself is pinned by tests/test_learned_reference.py:
at the initial model (the ES width-4 kernel fitted by polynomials, zero MLP
output, no correction) it reproduces the direct Eq. 7 sum of the oracle to
the width-4 kernel's accuracy.
"""
from __future__ import annotations

import numpy as np

W = 4
DEG = 7
K = DEG + 1
T = 2 * W * K
F = 6
H = 32
C = 6
SRC_TILE = 16
OUT_SCALE = 1e-3
BETA = 2.30 * W

# layout of the model vector (include/asfd.h)
SL_BASE = slice(0, T)
SL_W1 = slice(T, T + H * F)
SL_B1 = slice(SL_W1.stop, SL_W1.stop + H)
SL_W2 = slice(SL_B1.stop, SL_B1.stop + T * H)
SL_B2 = slice(SL_W2.stop, SL_W2.stop + T)
SL_DX = slice(SL_B2.stop, SL_B2.stop + C)
SL_DY = slice(SL_DX.stop, SL_DX.stop + C)
N_PARAMS = SL_DY.stop


def es(z, w=W, beta=BETA):
    u = 2.0 * np.asarray(z, np.float64) / w
    inside = np.abs(u) <= 1.0
    return np.where(inside, np.exp(beta * (np.sqrt(np.clip(1.0 - u * u, 0.0, None)) - 1.0)), 0.0)


def es_hat(xi, w=W, beta=BETA, nodes=400):
    """int_{-w/2}^{w/2} psi(z) exp(-i xi z) dz (real, even) by Gauss-Legendre."""
    x, wt = np.polynomial.legendre.leggauss(nodes)
    z = 0.25 * w * (x + 1.0)               # [0, w/2]
    wz = 0.25 * w * wt
    xi = np.asarray(xi, np.float64)
    return 2.0 * np.sum(wz[None, :] * es(z)[None, :] * np.cos(xi[:, None] * z[None, :]), axis=1)


def es_fit_table():
    """Least-squares fit of the ES taps by degree-7 polynomials in t = 2 dx - 1
    (numpy polyfit on Chebyshev nodes); same table for x and y."""
    t = np.cos(np.pi * (np.arange(256) + 0.5) / 256)
    dx = 0.5 * (t + 1.0)
    tab = np.zeros((2, W, K))
    for a in range(W):
        coef = np.polynomial.polynomial.polyfit(t, es(dx + a - 0.5 * W), DEG)
        tab[0, a] = coef
        tab[1, a] = coef
    return tab.ravel()


def initial_params():
    p = np.zeros(N_PARAMS)
    p[SL_BASE] = es_fit_table()
    return p


def _positions(g, d1, nfx, nfy):
    lam_z0 = g["lam"] * g["z0"]
    xt = (np.arange(g["n1x"]) - g["n1x"] // 2).astype(np.float64)
    yt = (np.arange(g["n1y"]) - g["n1y"] // 2).astype(np.float64)
    scale = g["z0"] / (g["z0"] - np.asarray(d1, np.float64))      # z0 / r0
    gx = g["p1x"] * g["p2x"] * nfx / lam_z0 * xt[None, :] * scale + 0.5 * nfx
    gy = g["p1y"] * g["p2y"] * nfy / lam_z0 * yt[:, None] * scale + 0.5 * nfy
    return gx, gy


def features(g, d1, nfx, nfy):
    """Per source tile (16 x 16 samples, row-major tiles): the six features."""
    gx, gy = _positions(g, d1, nfx, nfy)
    q = np.asarray(d1) / (g["z0"] - np.asarray(d1))
    n1y, n1x = gx.shape
    ntx = (n1x + SRC_TILE - 1) // SRC_TILE
    nty = (n1y + SRC_TILE - 1) // SRC_TILE
    out = np.zeros((nty * ntx, F))
    sx = np.full(gx.shape, np.nan)
    sx[:, :-1] = gx[:, 1:] - gx[:, :-1]
    sy = np.full(gy.shape, np.nan)
    sy[:-1, :] = gy[1:, :] - gy[:-1, :]
    for ty in range(nty):
        for tx in range(ntx):
            blk = (slice(ty * SRC_TILE, (ty + 1) * SRC_TILE), slice(tx * SRC_TILE, (tx + 1) * SRC_TILE))
            bsx = sx[blk][~np.isnan(sx[blk])]
            bsy = sy[blk][~np.isnan(sy[blk])]
            out[ty * ntx + tx] = [1.0,
                                  np.mean((gx[blk] - 0.5 * nfx) / (0.5 * nfx)),
                                  np.mean((gy[blk] - 0.5 * nfy) / (0.5 * nfy)),
                                  (np.mean(bsx) if bsx.size else 1.0) - 1.0,
                                  (np.mean(bsy) if bsy.size else 1.0) - 1.0,
                                  100.0 * np.mean(q[blk])]
    return out


def tables(params, feats):
    p = np.asarray(params, np.float64)
    w1 = p[SL_W1].reshape(H, F)
    w2 = p[SL_W2].reshape(T, H)
    h = np.tanh(feats @ w1.T + p[SL_B1][None, :])
    return p[SL_BASE][None, :] + OUT_SCALE * (h @ w2.T + p[SL_B2][None, :])


def _cheb_even(u):
    """T_2j(u) for j = 1..C, shape [len(u), C]."""
    u = np.asarray(u, np.float64)
    return np.stack([np.cos(2 * j * np.arccos(np.clip(u, -1, 1))) for j in range(1, C + 1)], axis=1)


def forward(g, u1, d1, params, sigma=2.0):
    """u2 [m2y, m2x] of the learned-kernel transform, FP64."""
    nfx = int(round(sigma * g["m2x"]))
    nfy = int(round(sigma * g["m2y"]))
    k = 2 * np.pi / g["lam"]
    d1 = np.asarray(d1, np.float64)
    n1y, n1x = d1.shape
    x1 = (np.arange(n1x) - n1x // 2) * g["p1x"]
    y1 = (np.arange(n1y) - n1y // 2) * g["p1y"]
    r0 = g["z0"] - d1
    c = np.asarray(u1, np.complex128) * np.exp(1j * k * d1) * np.exp(
        1j * k * (-d1 + (x1[None, :] ** 2 + y1[:, None] ** 2) / (2 * r0)))
    gx, gy = _positions(g, d1, nfx, nfy)
    l0x = np.ceil(gx - 0.5 * W)
    l0y = np.ceil(gy - 0.5 * W)
    tx = 2.0 * (l0x - (gx - 0.5 * W)) - 1.0
    ty = 2.0 * (l0y - (gy - 0.5 * W)) - 1.0
    tab = tables(params, features(g, d1, nfx, nfy)).reshape(-1, 2, W, K)
    ntx = (n1x + SRC_TILE - 1) // SRC_TILE
    tile = (np.arange(n1y)[:, None] // SRC_TILE) * ntx + np.arange(n1x)[None, :] // SRC_TILE
    b = np.zeros((nfy, nfx), np.complex128)
    px = [np.einsum("ijk,ijk->ij", tab[tile, 0, a, :], tx[..., None] ** np.arange(K))
          for a in range(W)]
    py = [np.einsum("ijk,ijk->ij", tab[tile, 1, bb, :], ty[..., None] ** np.arange(K))
          for bb in range(W)]
    for bb in range(W):
        rows = (l0y.astype(np.int64) + bb) % nfy
        for a in range(W):
            cols = (l0x.astype(np.int64) + a) % nfx
            np.add.at(b, (rows.ravel(), cols.ravel()), (c * px[a] * py[bb]).ravel())
    spec = np.fft.fft2(b)
    mpx = np.arange(g["m2x"]) - g["m2x"] // 2
    mpy = np.arange(g["m2y"]) - g["m2y"] // 2
    F2 = spec[np.ix_(mpy % nfy, mpx % nfx)]
    p = np.asarray(params, np.float64)
    corr_x = 1.0 + _cheb_even(2.0 * mpx / g["m2x"]) @ p[SL_DX]
    corr_y = 1.0 + _cheb_even(2.0 * mpy / g["m2y"]) @ p[SL_DY]
    dec_x = (-1.0) ** (mpx & 1) * corr_x / es_hat(2 * np.pi * mpx / nfx)
    dec_y = (-1.0) ** (mpy & 1) * corr_y / es_hat(2 * np.pi * mpy / nfy)
    x2 = mpx * g["p2x"]
    y2 = mpy * g["p2y"]
    outer = np.exp(1j * k * (g["z0"] + (x2[None, :] ** 2 + y2[:, None] ** 2) / (2 * g["z0"]))) / (
        1j * g["lam"] * g["z0"]) * g["p1x"] * g["p1y"]
    return outer * dec_y[:, None] * dec_x[None, :] * F2


def loss(u2, ref):
    return float(np.sum(np.abs(u2 - ref) ** 2) / np.sum(np.abs(ref) ** 2))
