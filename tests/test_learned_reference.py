"""Pins for the FP64 CPU reference of the learned-kernel forward map (CPU only).

* its ES transform matches adaptive quadrature (scipy) of the ES kernel;
* its polynomial fit reproduces the ES kernel taps;
* at the initial model (ES width 4 fitted by polynomials, zero MLP output,
  no deconvolution correction) the whole map reproduces the direct Eq. 7 sum
  of the oracle to the accuracy of a width-4 kernel at oversampling 2;
* the deconvolution correction equals the closed-form even Chebyshev series,
  the MLP's output bias is a shift of every tile's table, and the field is
  linear in one axis's tap tables.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
from oracle import learned_ref as R
from paper_1203_3583_gb300 import workloads as W


def test_es_hat_matches_adaptive_quadrature():
    integrate = pytest.importorskip("scipy.integrate")
    for xi in (0.0, 0.7, 1.5, np.pi / 2):
        ref = integrate.quad(lambda z: float(R.es(z)) * np.cos(xi * z), -2.0, 2.0, limit=200,
                             epsabs=1e-14, epsrel=1e-13)[0]
        assert abs(R.es_hat(np.array([xi]))[0] - ref) < 1e-10 * max(1.0, abs(ref))


def test_polynomial_fit_of_es_taps():
    tab = R.es_fit_table().reshape(2, R.W, R.K)
    dx = np.linspace(0.0, 0.999, 101)
    for a in range(R.W):
        fit = np.polynomial.polynomial.polyval(2 * dx - 1, tab[0, a])
        assert np.max(np.abs(fit - R.es(dx + a - 2.0))) < 2e-4


@pytest.mark.parametrize("name", ["sinusoid64", "ragged"])
def test_initial_model_reproduces_eq7(name):
    rng = np.random.default_rng(51)
    if name == "ragged":
        g = W.geometry(50, 38, 10e-6, 7e-6, 64, 32, 12e-6, 9e-6, 532e-9, 0.04)
        u1 = rng.standard_normal((38, 50)) + 1j * rng.standard_normal((38, 50))
        d1 = W.surface_smooth_random(g, rng, 4.0, 60e-6) - 30e-6
    else:
        g, _, d1 = W.make(name)
        u1 = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))
    u2 = R.forward(g, u1, d1, R.initial_params())
    ref = oracle.eq7(g, u1, d1)
    err = np.linalg.norm(u2 - ref) / np.linalg.norm(ref)
    assert err < 5e-3, err


def _small_case():
    rng = np.random.default_rng(52)
    g = W.geometry(40, 36, 10e-6, 9e-6, 32, 32, 11e-6, 10e-6, 633e-9, 0.05)
    u1 = rng.standard_normal((36, 40)) + 1j * rng.standard_normal((36, 40))
    d1 = W.surface_smooth_random(g, rng, 4.0, 40e-6) - 20e-6
    return g, u1, d1


def test_deconvolution_correction_is_the_even_chebyshev_series():
    """corr(u) = 1 + d1 T2(u) + d2 T4(u) with the closed forms T2 = 2u^2 - 1 and
    T4 = 8u^4 - 8u^2 + 1, u = 2 m'/M, applied per axis to the output."""
    g, u1, d1 = _small_case()
    p0 = R.initial_params()
    p = p0.copy()
    p[R.SL_DX.start:R.SL_DX.start + 2] = [0.03, -0.02]
    p[R.SL_DY.start:R.SL_DY.start + 2] = [-0.01, 0.04]
    base = R.forward(g, u1, d1, p0)
    got = R.forward(g, u1, d1, p)
    ux = 2.0 * (np.arange(g["m2x"]) - g["m2x"] // 2) / g["m2x"]
    uy = 2.0 * (np.arange(g["m2y"]) - g["m2y"] // 2) / g["m2y"]
    cx = 1 + 0.03 * (2 * ux ** 2 - 1) - 0.02 * (8 * ux ** 4 - 8 * ux ** 2 + 1)
    cy = 1 - 0.01 * (2 * uy ** 2 - 1) + 0.04 * (8 * uy ** 4 - 8 * uy ** 2 + 1)
    want = base * cy[:, None] * cx[None, :]
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def test_mlp_output_bias_moves_every_tile_table():
    """With the hidden-to-output weights zero the MLP adds OUT_SCALE * b2 to
    every tile's table, which must equal moving the shared base by that much;
    a nonzero hidden layer then changes the field (the tables depend on it)."""
    g, u1, d1 = _small_case()
    rng = np.random.default_rng(53)
    b2 = rng.standard_normal(R.T)
    p_bias = R.initial_params()
    p_bias[R.SL_B2] = b2
    p_bias[R.SL_W1] = rng.standard_normal(R.H * R.F)   # hidden layer present, output weights 0
    p_base = R.initial_params()
    p_base[R.SL_BASE] += R.OUT_SCALE * b2
    a = R.forward(g, u1, d1, p_bias)
    b = R.forward(g, u1, d1, p_base)
    assert np.max(np.abs(a - b)) <= 1e-12 * np.max(np.abs(b))
    p_w2 = p_bias.copy()
    p_w2[R.SL_W2] = rng.standard_normal(R.T * R.H)
    c = R.forward(g, u1, d1, p_w2)
    assert np.linalg.norm(c - a) > 1e-6 * np.linalg.norm(a)


def test_table_is_linear_in_the_spread():
    """The field is linear in the tap polynomials of one axis: doubling every
    x-axis tap table doubles u2."""
    g, u1, d1 = _small_case()
    p = R.initial_params()
    tab = p[R.SL_BASE].reshape(2, R.W, R.K)
    tab[0] *= 2.0
    p[R.SL_BASE] = tab.ravel()
    base = R.forward(g, u1, d1, R.initial_params())
    got = R.forward(g, u1, d1, p)
    assert np.max(np.abs(got - 2.0 * base)) <= 1e-12 * np.max(np.abs(base))
