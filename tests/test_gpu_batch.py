"""Batched persistent kernel (all surfaces in one cooperative launch, CUDA graph).

The 24-surface RGB workload (sizes 256^2..2048^2, 450/532/633 nm, z0 in
0.05-0.3 m, sinusoidal or smooth random surfaces): every surface's output
equals that surface's own plan, and matches the FP64 oracle on seeded
destination points; a second launch with new fields reuses the graph.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelBatch, FresnelPlan  # noqa: E402

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


@pytest.fixture(scope="module")
def rgb_batch():
    items = W.make_batch()
    with FresnelBatch([(g, d1) for g, _, d1 in items]) as b:
        u1 = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
        out = b.execute(u1)
        torch.cuda.synchronize()
        info = b.info()
        out_np = [o.cpu().numpy() for o in out]
        # second launch with new fields through the same graph
        rng = np.random.default_rng(9)
        u1b = [torch.as_tensor(W.field_random_amp_phase(g, rng), device="cuda") for g, _, _ in items]
        out_b = [o.cpu().numpy() for o in b.execute(u1b)]
        torch.cuda.synchronize()
    return items, out_np, info, [u.cpu().numpy() for u in u1b], out_b


def test_batch_info(rgb_batch):
    items, _, info, _, _ = rgb_batch
    assert info["surfaces"] == 24
    assert info["source_samples"] == sum(g["n1x"] * g["n1y"] for g, _, _ in items)
    assert info["blocks"] >= 1


def test_batch_equals_individual_plans(rgb_batch):
    items, out, _, u1b, out_b = rgb_batch
    for i, (g, u1, d1) in enumerate(items):
        with FresnelPlan(g, d1) as p:
            ref = p.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
            ref_b = p.execute(torch.as_tensor(u1b[i], device="cuda")).cpu().numpy()
        # identical arithmetic except the order of shared-memory float atomics
        # (surfaces on the atomic spreading path) and FFT line grouping
        assert rel_l2(out[i], ref) < 5e-6, i
        assert rel_l2(out_b[i], ref_b) < 5e-6, i


def test_batch_matches_oracle(rgb_batch):
    """512 seeded destination points per surface."""
    items, out, _, _, _ = rgb_batch
    for i, (g, u1, d1) in enumerate(items):
        pts = W.sample_points(g, 512, seed=400 + i)
        ref = oracle.eq7(g, u1, d1, points=pts)
        err = rel_l2(out[i][pts[1], pts[0]], ref)
        assert err < 1e-5, (i, err)


def test_deterministic_batch_equals_individual_plans():
    """With deterministic=True every surface takes atomic-free spreading (or
    shared-memory atomics where the map needs them); the batch still equals
    the surfaces' own plans."""
    items = W.make_batch()[:8]
    with FresnelBatch([(g, d1) for g, _, d1 in items], deterministic=True) as b:
        out = b.execute([torch.as_tensor(u, device="cuda") for _, u, _ in items])
        torch.cuda.synchronize()
        got = [o.cpu().numpy() for o in out]
    for i, (g, u1, d1) in enumerate(items):
        with FresnelPlan(g, d1, deterministic=True) as p:
            ref = p.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
        assert rel_l2(got[i], ref) < 5e-6, i
