"""Batched transform, in both schedules: the surfaces' kernels on the batch's
streams (the default, CUDA graph per set of field pointers) and one
persistent cooperative launch (CUDA graph).

The 24-surface RGB workload (sizes 256^2..2048^2, 450/532/633 nm, z0 in
0.05-0.3 m, sinusoidal or smooth random surfaces): every surface's output
equals that surface's own plan, and matches the FP64 oracle on seeded
destination points; later launches with new fields go through the graph.
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


@pytest.fixture(scope="module", params=["streams", "persistent"])
def rgb_batch(request):
    items = W.make_batch()
    with FresnelBatch([(g, d1) for g, _, d1 in items]) as b:
        b.set_schedule(request.param)
        u1 = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
        out = b.execute(u1)
        torch.cuda.synchronize()
        out_np = [o.cpu().numpy() for o in out]
        # later launches with new fields: new pointers (a new capture), then
        # the same pointers with new contents (a replay)
        rng = np.random.default_rng(9)
        u1b = [torch.as_tensor(W.field_random_amp_phase(g, rng), device="cuda") for g, _, _ in items]
        outb = [torch.empty_like(o) for o in out]
        b.execute(u1b, out=outb)
        for u in u1b:
            u.mul_(1j)
        b.execute(u1b, out=outb)
        torch.cuda.synchronize()
        info = b.info()
        out_b = [o.cpu().numpy() for o in outb]
    return items, out_np, info, [u.cpu().numpy() for u in u1b], out_b


def test_batch_info(rgb_batch):
    items, _, info, _, _ = rgb_batch
    assert info["surfaces"] == 24
    assert info["source_samples"] == sum(g["n1x"] * g["n1y"] for g, _, _ in items)
    assert info["persistent_ok"] == 1 and info["blocks"] >= 1
    assert info["graph"] == 1
    assert info["streams"] == 16


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


def test_mixed_widths_batch_streams_only():
    """Surfaces with different kernel widths (and a width outside 4..8) form a
    valid batch on the stream schedule; the persistent schedule is refused."""
    items = W.make_batch()[:4]
    widths = [5, 7, 3, 9]
    params = [capi.make_params(g, kernel_width=w) for (g, _, _), w in zip(items, widths)]
    d1s = [torch.as_tensor(d1, device="cuda") for _, _, d1 in items]
    handle = capi.asfd_batch_create(params, d1s)
    try:
        info = capi.asfd_batch_get_info(handle)
        assert info["persistent_ok"] == 0 and info["schedule"] == 0
        with pytest.raises(capi.AsfdError):
            capi.asfd_batch_set_schedule(handle, "persistent")
        u1 = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
        outs = [torch.empty((g["m2y"], g["m2x"]), dtype=torch.complex64, device="cuda")
                for g, _, _ in items]
        for _ in range(3):  # direct, capture, replay
            capi.asfd_batch_execute(handle, u1, outs)
        torch.cuda.synchronize()
        for (g, u, d1), w, o in zip(items, widths, outs):
            with FresnelPlan(g, d1, kernel_width=w) as p:
                ref = p.execute(torch.as_tensor(u, device="cuda")).cpu().numpy()
            assert rel_l2(o.cpu().numpy(), ref) < 5e-6, w
    finally:
        capi.asfd_batch_destroy(handle)


def test_schedule_switch_keeps_results():
    """Streams, then persistent, then streams again on one batch: the
    persistent kernel leaves the dense surfaces' bands as its row stage read
    them, and the stream schedule starts its band state over."""
    items = W.make_batch()[:6]
    u1 = [torch.as_tensor(u, device="cuda") for _, u, _ in items]
    with FresnelBatch([(g, d1) for g, _, d1 in items]) as b:
        ref = [o.cpu().numpy() for o in b.execute(u1)]
        outs = [torch.empty_like(torch.as_tensor(r, device="cuda")) for r in ref]
        for sched in ("persistent", "streams", "persistent", "streams"):
            b.set_schedule(sched)
            for _ in range(3):
                b.execute(u1, out=outs)
            torch.cuda.synchronize()
            for i, o in enumerate(outs):
                assert rel_l2(o.cpu().numpy(), ref[i]) < 5e-6, (sched, i)
