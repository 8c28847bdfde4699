"""Pins for the FP64 CPU reference of the learned-kernel forward map (CPU only).

* its ES transform matches adaptive quadrature (scipy) of the ES kernel;
* its polynomial fit reproduces the ES kernel taps;
* at the initial model (ES width 4 fitted by polynomials, zero MLP output,
  no deconvolution correction) the whole map reproduces the direct Eq. 7 sum
  of the oracle to the accuracy of a width-4 kernel at oversampling 2.
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
