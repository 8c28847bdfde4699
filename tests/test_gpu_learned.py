"""Learned spreading kernel on the GPU against the FP64 CPU reference.

* forward: the library's learned-kernel transform equals the CPU reference
  of the same model (oracle/learned_ref.py) for a model with per-tile
  variation (random MLP weights), including ragged source tiles;
* training gradients: asfd_learned_gradient (forward, loss, adjoint FFT
  passes, table / MLP / deconvolution gradient kernels) equals central finite
  differences of the CPU reference's loss, parameter by parameter;
* gain: a model trained by the library's own kernels beats the ES kernel at
  the same width 4 on held-out surfaces, checked against the oracle.
"""
from __future__ import annotations

import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import learned_ref as R  # noqa: E402
from paper_1203_3583_gb300 import capi, learned as L, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_3583_gb300 import _build
    capi.load(_build.build())


def _case(name):
    rng = np.random.default_rng(61)
    if name == "ragged":
        g = W.geometry(50, 38, 10e-6, 7e-6, 64, 32, 12e-6, 9e-6, 532e-9, 0.04)
        d1 = W.surface_smooth_random(g, rng, 4.0, 60e-6) - 30e-6
    else:
        g, _, d1 = W.make("sinusoid64")
    u1 = (rng.standard_normal(d1.shape) + 1j * rng.standard_normal(d1.shape)).astype(np.complex64)
    return g, u1, d1


def _perturbed_params(plan, seed):
    rng = np.random.default_rng(seed)
    p = capi.asfd_learned_get_params(plan.handle).astype(np.float64)
    p[R.SL_W1] = rng.normal(0, 0.5, R.H * R.F)
    p[R.SL_B1] = rng.normal(0, 0.2, R.H)
    p[R.SL_W2] = rng.normal(0, 2.0, R.T * R.H)
    p[R.SL_B2] = rng.normal(0, 2.0, R.T)
    p[R.SL_DX] = rng.normal(0, 1e-3, R.C)
    p[R.SL_DY] = rng.normal(0, 1e-3, R.C)
    p32 = p.astype(np.float32)
    capi.asfd_learned_set_params(plan.handle, p32)
    return p32.astype(np.float64)


@pytest.mark.parametrize("name", ["sinusoid64", "ragged"])
def test_learned_forward_matches_cpu_reference(name):
    g, u1, d1 = _case(name)
    with FresnelPlan(g, d1, kind="learned") as plan:
        params = _perturbed_params(plan, 62)
        out = plan.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
    ref = R.forward(g, u1, d1, params)
    err = np.linalg.norm(out - ref) / np.linalg.norm(ref)
    assert err < 2e-5, err


def test_learned_gradient_matches_cpu_finite_differences():
    g, u1, d1 = _case("sinusoid64")
    target = oracle.eq7(g, u1, d1)
    with FresnelPlan(g, d1, kind="learned") as plan:
        params = _perturbed_params(plan, 63)
        grad, loss = capi.asfd_learned_gradient(plan.handle, torch.as_tensor(u1, device="cuda"),
                                                torch.as_tensor(target.astype(np.complex64),
                                                                device="cuda"),
                                                plan.shape1, plan.shape2)
    assert abs(loss - R.loss(R.forward(g, u1, d1, params), target)) < 1e-3 * loss
    rng = np.random.default_rng(64)
    idx = np.concatenate([
        np.arange(R.SL_BASE.start, R.SL_BASE.stop),
        rng.choice(np.arange(R.SL_W1.start, R.SL_W1.stop), 12, replace=False),
        rng.choice(np.arange(R.SL_B1.start, R.SL_B1.stop), 6, replace=False),
        rng.choice(np.arange(R.SL_W2.start, R.SL_W2.stop), 24, replace=False),
        rng.choice(np.arange(R.SL_B2.start, R.SL_B2.stop), 12, replace=False),
        np.arange(R.SL_DX.start, R.SL_DY.stop)])
    fd = np.empty(idx.size)
    for j, i in enumerate(idx):
        h = 1e-4 * max(1.0, abs(params[i]))
        pp = params.copy()
        pm = params.copy()
        pp[i] += h
        pm[i] -= h
        fd[j] = (R.loss(R.forward(g, u1, d1, pp), target) -
                 R.loss(R.forward(g, u1, d1, pm), target)) / (2 * h)
    ana = grad[idx].astype(np.float64)
    err = np.linalg.norm(ana - fd) / np.linalg.norm(fd)
    assert err < 3e-3, err
    # every parameter block carries signal (no block silently zero)
    for sl in (R.SL_BASE, R.SL_W1, R.SL_B1, R.SL_W2, R.SL_B2, R.SL_DX, R.SL_DY):
        assert np.any(grad[sl] != 0.0)


def test_trained_model_beats_es_at_width_4():
    pairs = L.train_set(surfaces=4, fields=2, seed=300)
    model, losses = L.train_model(pairs)
    assert math.sqrt(losses[-1]) < math.sqrt(losses[0])
    g, u1, d1 = L.train_set(surfaces=1, fields=1, seed=700)[0]
    pts = W.sample_points(g, 512, seed=701)
    ref = oracle.eq7(g, u1, d1, points=pts)
    with FresnelPlan(g, d1, kind="learned") as p:
        model.apply_to(p)
        lw = p.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()[pts[1], pts[0]]
    with FresnelPlan(g, d1, kernel_width=4) as p:
        es4 = p.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()[pts[1], pts[0]]
    e_learned = np.linalg.norm(lw - ref) / np.linalg.norm(ref)
    e_es4 = np.linalg.norm(es4 - ref) / np.linalg.norm(ref)
    assert e_learned < 0.7 * e_es4, (e_learned, e_es4)
