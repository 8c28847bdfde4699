"""Failure paths on the GPU without faulting it: the library's allocation
hook (asfd_debug_fail_allocations) refuses the device allocations of 2D plans
one after another; every refusal must come back as ASFD_ERR_NOMEM with no
buffer left behind (asfd_debug_live_buffers), and the plan finally built must
still match the oracle.  Nothing here makes a kernel fail."""
from __future__ import annotations

import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelBatch, FresnelPlan  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_3583_gb300 import _build
    return capi.load(_build.build())


def build_with_failures(lib, make, limit=200):
    """Calls make() with 0, 1, 2, ... allocations allowed; returns the object
    and the number of allocations it needed.  Plans of earlier tests that
    only the cycle collector would free are collected first, and collection
    is paused meanwhile, so that the live-buffer count moves only with make()."""
    gc.collect()
    gc.disable()
    base = lib.asfd_debug_live_buffers()
    try:
        for k in range(limit):
            lib.asfd_debug_fail_allocations(k)
            try:
                obj = make()
            except capi.AsfdError as e:
                assert e.status == capi.ASFD_ERR_NOMEM, str(e)
                assert lib.asfd_debug_live_buffers() == base, f"buffers left after failure {k}"
                continue
            return obj, k
    finally:
        lib.asfd_debug_fail_allocations(-1)
        gc.enable()
    raise AssertionError("still failing after the allocation limit")


@pytest.mark.parametrize("deterministic", [False, True])
def test_plan_allocation_failures_leave_nothing_behind(lib, deterministic):
    g, u1, d1 = W.make("sinusoid64")
    gc.collect()
    base = lib.asfd_debug_live_buffers()
    plan, needed = build_with_failures(lib, lambda: FresnelPlan(g, d1, deterministic=deterministic))
    assert needed > 0
    with plan:
        assert lib.asfd_debug_live_buffers() > base
        out = plan.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
    assert lib.asfd_debug_live_buffers() == base
    ref = oracle.eq7(g, u1, d1)
    err = float(np.linalg.norm(out - ref) / np.linalg.norm(ref))
    assert err < 1e-5, err


def test_batch_allocation_failures_leave_nothing_behind(lib):
    g, u1, d1 = W.make("sinusoid64")
    rng = np.random.default_rng(71)
    u1b = (rng.standard_normal(u1.shape) + 1j * rng.standard_normal(u1.shape)).astype(np.complex64)
    items = [(g, u1, d1), (g, u1b, 0.5 * d1)]
    gc.collect()
    base = lib.asfd_debug_live_buffers()
    batch, needed = build_with_failures(lib, lambda: FresnelBatch([(g, d1) for g, _, d1 in items]))
    assert needed > 0
    with batch:
        outs = batch.execute([torch.as_tensor(u, device="cuda") for _, u, _ in items])
        got = [o.cpu().numpy() for o in outs]
    assert lib.asfd_debug_live_buffers() == base
    for (g, u1, d1), out in zip(items, got):
        ref = oracle.eq7(g, u1, d1)
        assert float(np.linalg.norm(out - ref) / np.linalg.norm(ref)) < 1e-5


def test_hook_off_by_default(lib):
    g, u1, d1 = W.make("sinusoid64")
    with FresnelPlan(g, d1):
        pass


def test_work_buffer_allocation_failures(lib):
    """The work buffers a plan allocates on first use (fine grid and row
    buffer at the first execution, the u1/u2 staging at the first
    asfd_execute_host on pageable buffers) go through the same hook: each refusal returns
    ASFD_ERR_NOMEM, leaves no buffer behind and leaves the plan usable."""
    g, u1, d1 = W.make("sinusoid64")
    gc.collect()
    base = lib.asfd_debug_live_buffers()
    u1_t = torch.as_tensor(u1, device="cuda")
    # pageable host buffers: asfd_execute_host stages them through device copies
    host_in = torch.as_tensor(u1).clone()
    host_out = torch.empty((g["m2y"], g["m2x"]), dtype=torch.complex64)
    ref = oracle.eq7(g, u1, d1)
    with FresnelPlan(g, d1) as plan:
        tables = lib.asfd_debug_live_buffers()
        for k in (0, 1):  # refuse the fine grid, then the row buffer
            lib.asfd_debug_fail_allocations(k)
            try:
                with pytest.raises(capi.AsfdError) as ei:
                    plan.execute(u1_t)
            finally:
                lib.asfd_debug_fail_allocations(-1)
            assert ei.value.status == capi.ASFD_ERR_NOMEM
            assert lib.asfd_debug_live_buffers() == tables
        # refuse the grid, the row buffer, then (with those two in place) the
        # staging of u1, then the staging of u2
        for k, kept in ((0, 0), (1, 0), (2, 2), (1, 2)):
            lib.asfd_debug_fail_allocations(k)
            try:
                with pytest.raises(capi.AsfdError) as ei:
                    plan.execute_host(host_in, host_out)
            finally:
                lib.asfd_debug_fail_allocations(-1)
            assert ei.value.status == capi.ASFD_ERR_NOMEM
            # the transform's pair stays once allocated; a refused pair leaves nothing
            assert lib.asfd_debug_live_buffers() == tables + kept
        plan.execute_host(host_in, host_out)
        assert lib.asfd_debug_live_buffers() == tables + 4
        out = plan.execute(u1_t).cpu().numpy()
    assert lib.asfd_debug_live_buffers() == base
    for x in (out, host_out.numpy()):
        assert float(np.linalg.norm(x - ref) / np.linalg.norm(ref)) < 1e-5
