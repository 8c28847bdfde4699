"""Learned spreading kernel on the GPU against the FP64 CPU reference.

* forward: the library's learned-kernel transform equals the CPU reference
  of the same model (oracle/learned_ref.py) for a model with per-tile
  variation (random MLP weights), including ragged source tiles;
* training gradients: asfd_learned_gradient (forward, loss, adjoint FFT
  passes, table / MLP / deconvolution gradient kernels) equals central finite
  differences of the CPU reference's loss, parameter by parameter;
* accuracy: a model trained by the library's own kernels on held-out
  surfaces reaches the width-4 floor (the best any width-4 gridding can do,
  oracle/learned_floor.py) on the 2048^2 workload against the oracle, about
  4x below the ES kernel of the same width.
"""
from __future__ import annotations

import math
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from oracle import learned_ref as R  # noqa: E402
from paper_1203_3583_gb300 import capi, learned as L, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan  # noqa: E402
from tests.oracle_cache import sampled  # noqa: E402

pytestmark = pytest.mark.gpu

GOLDEN_FLOOR = os.path.join(os.path.dirname(__file__), "golden", "learned_floor_sigma2.txt")


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


def _width4_floor():
    """The smallest relative L2 error any width-4 gridding reaches at sigma = 2
    on random-phase samples (2D), as written by tests/golden/make_learned_floor.py
    from the oracle (pinned in tests/test_learned_floor_cpu.py)."""
    for line in open(GOLDEN_FLOOR):
        if line.strip() and not line.startswith("#") and line.split()[0] == "4":
            return float(line.split()[2])
    raise AssertionError("no width-4 row in " + GOLDEN_FLOOR)


def test_learned_reaches_width4_floor_on_smooth_random2048():
    """The model trained by the library's own kernels (Adam on the GPU, two
    held-out surfaces of the 2048^2 recipe) against the FP64 oracle of Eq. 7
    on 4096 seeded points of the 2048^2 workload itself.

    The target of 1e-4 at width 4 lies below the width-4 floor (2.71e-4: no
    tap table and no per-mode correction of width 4 does better on
    random-phase samples at sigma = 2), so the bar here is the floor: within
    15 % above it, never meaningfully below it, and at least 3x better than
    the ES kernel of the same width on the same points."""
    floor = _width4_floor()
    pairs = L.train_set(seed=300)
    model, losses = L.train_model(pairs)
    assert math.sqrt(losses[-1]) < 0.4 * math.sqrt(losses[0])
    g, u1, d1, pts, ref = sampled("smooth_random2048", 4096, 103)
    u1_t = torch.as_tensor(u1, device="cuda")
    with FresnelPlan(g, d1, kind="learned") as p:
        model.apply_to(p)
        lw = p.execute(u1_t).cpu().numpy()[pts[1], pts[0]]
    with FresnelPlan(g, d1, kernel_width=4) as p:
        es4 = p.execute(u1_t).cpu().numpy()[pts[1], pts[0]]
    e_learned = np.linalg.norm(lw - ref) / np.linalg.norm(ref)
    e_es4 = np.linalg.norm(es4 - ref) / np.linalg.norm(ref)
    assert 0.9 * floor < e_learned < 1.15 * floor, (e_learned, floor)
    assert e_learned < e_es4 / 3.0, (e_learned, e_es4)
