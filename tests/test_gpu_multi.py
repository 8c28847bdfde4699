"""Several surfaces summed at one destination (asfd_multi_execute): source
grids placed off the axis (asfd_params offset_x/y) against the oracle, the
shared-grid sum against the sum of the surfaces' own transforms and against
the oracle, and the compatibility checks."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan, direct_sum, multi_execute  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_3583_gb300 import _build
    capi.load(_build.build())


def rel_l2(a, b):
    a = np.asarray(a, np.complex128).ravel()
    b = np.asarray(b, np.complex128).ravel()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("deterministic", [False, True])
def test_offset_surface_matches_oracle(deterministic):
    g, u1, d1 = W.make("sinusoid64")
    g = dict(g, ox=70e-6, oy=-130e-6)
    rng = np.random.default_rng(61)
    u = (rng.standard_normal(u1.shape) + 1j * rng.standard_normal(u1.shape)).astype(np.complex64)
    with FresnelPlan(g, d1, deterministic=deterministic) as p:
        out = p.execute(torch.as_tensor(u, device="cuda")).cpu().numpy()
    assert rel_l2(out, oracle.eq7(g, u, d1)) < 1e-5


def test_offset_direct_sum_matches_oracle():
    g, u1, d1 = W.make("spherical_cap1024")
    g = dict(g, ox=-0.7e-3, oy=0.4e-3)
    pts = W.sample_points(g, 24, seed=62)
    got = direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), 7, pts).cpu().numpy()
    assert rel_l2(got, oracle.eq7(g, u1, d1, points=pts)) < 2e-6


def test_multi_surface_sum():
    items = W.make_multi()
    plans = [FresnelPlan(g, d1) for g, _, d1 in items]
    try:
        u1s = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
        total = multi_execute(plans, u1s).cpu().numpy().astype(np.complex128)
        each = sum(p.execute(u).cpu().numpy().astype(np.complex128) for p, u in zip(plans, u1s))
    finally:
        for p in plans:
            p.close()
    assert rel_l2(total, each) < 2e-6
    g0 = items[0][0]
    pts = W.sample_points(g0, 96, seed=63)
    ref = sum(oracle.eq7(g, u, d1, points=pts) for g, u, d1 in items)
    assert rel_l2(total[pts[1], pts[0]], ref) < 1e-5


def test_multi_surface_rejects_mismatched_destination():
    items = W.make_multi()[:2]
    g1 = dict(items[1][0], z0=0.25)
    plans = [FresnelPlan(items[0][0], items[0][2]), FresnelPlan(g1, items[1][2])]
    try:
        u1s = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
        with pytest.raises(capi.AsfdError):
            multi_execute(plans, u1s)
    finally:
        for p in plans:
            p.close()


def test_multi_surface_rejects_deterministic_plans():
    g, u1, d1 = W.make("sinusoid64")
    plans = [FresnelPlan(g, d1, deterministic=True), FresnelPlan(g, d1, deterministic=True)]
    try:
        u = torch.as_tensor(u1, device="cuda")
        with pytest.raises(capi.AsfdError):
            multi_execute(plans, [u, u])
    finally:
        for p in plans:
            p.close()
