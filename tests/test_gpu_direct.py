"""GPU direct sums of Eq. 7, Eq. 5 and Eq. 2 (asfd_direct_sum) against the FP64
oracle on the same seeded inputs, and the NUFFT path against the GPU Eq. 7
sum at full size on sampled points."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan, direct_sum  # noqa: E402

pytestmark = pytest.mark.gpu

# FP32 sine/cosine of an exactly reduced FP64 phase and FP32 products, FP64 sums
TOL_DIRECT = 2e-6


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


ORACLE = {7: oracle.eq7, 5: oracle.eq5, 2: oracle.eq2}


@pytest.mark.parametrize("form", [7, 5, 2])
def test_direct_sum_full_grid_sinusoid64(form):
    g, u1, d1 = W.make("sinusoid64")
    my, mx = np.meshgrid(np.arange(g["m2y"]), np.arange(g["m2x"]), indexing="ij")
    pts = (mx.ravel(), my.ravel())
    got = direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), form, pts).cpu().numpy()
    ref = ORACLE[form](g, u1, d1, points=pts)
    assert rel_l2(got, ref) < TOL_DIRECT, form


@pytest.mark.parametrize("form", [7, 5, 2])
def test_direct_sum_sampled_spherical_cap1024(form):
    g, u1, d1 = W.make("spherical_cap1024")
    pts = W.sample_points(g, 67, seed=300 + form)  # a ragged tail of the 8-point blocks
    got = direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), form, pts).cpu().numpy()
    ref = ORACLE[form](g, u1, d1, points=pts)
    assert rel_l2(got, ref) < TOL_DIRECT, form


def test_nufft_matches_direct_eq7_at_2048():
    g, u1, d1 = W.make("smooth_random2048")
    pts = W.sample_points(g, 256, seed=310)
    u = torch.as_tensor(u1, device="cuda")
    with FresnelPlan(g, d1) as plan:
        out = plan.execute(u).cpu().numpy()
    got = direct_sum(g, d1, u, 7, pts).cpu().numpy()
    assert rel_l2(out[pts[1], pts[0]], got) < 1e-5


def test_direct_sum_rejects_unknown_form():
    g, u1, d1 = W.make("sinusoid64")
    with pytest.raises(capi.AsfdError):
        direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), 3, ([0], [0]))


def test_direct_sum_empty_point_list():
    g, u1, d1 = W.make("sinusoid64")
    out = direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), 7,
                     (np.zeros(0, np.int32), np.zeros(0, np.int32)))
    assert out.numel() == 0


@pytest.mark.parametrize("form", [7, 5, 2])
def test_direct_sum_tilted_incidence(form):
    g, u1, d1 = W.make("spherical_cap1024")
    g = dict(g, sx=-0.008, sy=0.013)
    pts = W.sample_points(g, 40, seed=320 + form)
    got = direct_sum(g, d1, torch.as_tensor(u1, device="cuda"), form, pts).cpu().numpy()
    ref = ORACLE[form](g, u1, d1, points=pts)
    assert rel_l2(got, ref) < TOL_DIRECT, form
