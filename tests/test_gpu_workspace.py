"""Caller-owned workspace (asfd_workspace_bytes / asfd_set_workspace).

The plan's work buffers (fine grid, row buffer, host-execute staging, learned
training buffers) come from one uint8 tensor of PyTorch's caching allocator.
With the allocation hook refusing every device allocation of the library, the
forward transform (device and host buffers), the adjoint and a learned
training step still run, the plan holds only its tables, and the results
match the FP64 oracle of Eq. 7 (Sec. 2) at the ES bar of 1e-5."""
from __future__ import annotations

import ctypes
import gc

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_3583_gb300 import _build
    return capi.load(_build.build())


def rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("deterministic", [False, True])
def test_workspace_plan_allocates_nothing_and_matches_oracle(lib, deterministic):
    g, u1, d1 = W.make("spherical_cap1024", scale=8)
    gc.collect()
    plan = FresnelPlan(g, d1, deterministic=deterministic)
    try:
        tables = lib.asfd_debug_live_buffers()
        info0 = plan.info()
        ws = torch.empty(capi.asfd_workspace_bytes(plan.params), dtype=torch.uint8, device="cuda")
        plan.set_workspace(ws)
        lib.asfd_debug_fail_allocations(0)  # every further library allocation fails
        try:
            u1_t = torch.as_tensor(u1, device="cuda")
            out = plan.execute(u1_t)
            host = torch.empty(plan.shape2, dtype=torch.complex64)  # pageable: staged
            plan.execute_host(torch.as_tensor(u1).clone(), host)
            gu2 = torch.as_tensor(np.conj(np.asarray(out.cpu())), device="cuda")
            gu1 = torch.empty_like(u1_t)
            gd1 = torch.empty(plan.shape1, dtype=torch.float32, device="cuda")
            plan.adjoint(u1_t, gu2, gu1, gd1)
            torch.cuda.synchronize()
        finally:
            lib.asfd_debug_fail_allocations(-1)
        assert lib.asfd_debug_live_buffers() == tables
        assert plan.info()["device_bytes"] == info0["device_bytes"]
        got = out.cpu().numpy()
        pts = W.sample_points(g, 512, seed=11)
        ref = oracle.eq7(g, u1, d1, points=pts)
        assert rel(got[pts[1], pts[0]], ref) < 1e-5
        assert np.array_equal(host.numpy(), got) or rel(host.numpy(), got) < 1e-6
        assert np.isfinite(gu1.cpu().numpy()).all() and np.isfinite(gd1.cpu().numpy()).all()
    finally:
        plan.close()


def test_workspace_replaces_own_buffers_and_detaches(lib):
    g, u1, d1 = W.make("sinusoid64")
    gc.collect()
    base = lib.asfd_debug_live_buffers()
    with FresnelPlan(g, d1) as plan:
        tables = lib.asfd_debug_live_buffers() - base
        u1_t = torch.as_tensor(u1, device="cuda")
        a = plan.execute(u1_t).cpu().numpy()
        # the first execution allocated the fine grid and the row buffer
        assert lib.asfd_debug_live_buffers() - base == tables + 2
        host = torch.empty(plan.shape2, dtype=torch.complex64)  # pageable: staged
        plan.execute_host(torch.as_tensor(u1).clone(), host)
        assert lib.asfd_debug_live_buffers() - base == tables + 4
        plan.set_workspace(torch.empty(capi.asfd_workspace_bytes(plan.params), dtype=torch.uint8,
                                       device="cuda"))
        assert lib.asfd_debug_live_buffers() - base == tables
        b = plan.execute(u1_t).cpu().numpy()
        plan.set_workspace(None)
        assert lib.asfd_debug_live_buffers() - base == tables
        c = plan.execute(u1_t).cpu().numpy()
        assert lib.asfd_debug_live_buffers() - base == tables + 2
    assert lib.asfd_debug_live_buffers() == base
    ref = oracle.eq7(g, u1, d1)
    for x in (a, b, c, host.numpy()):
        assert rel(x, ref) < 1e-5


def test_workspace_argument_checks(lib):
    g, u1, d1 = W.make("sinusoid64")
    with FresnelPlan(g, d1) as plan:
        need = capi.asfd_workspace_bytes(plan.params)
        ws = torch.empty(need + 256, dtype=torch.uint8, device="cuda")
        h = plan.handle
        assert lib.asfd_set_workspace(h, ctypes.c_void_p(ws.data_ptr()), need - 1) == 1
        assert b"smaller" in lib.asfd_last_error()
        assert lib.asfd_set_workspace(h, ctypes.c_void_p(ws.data_ptr() + 16), need) == 1
        assert b"aligned" in lib.asfd_last_error()
        hostbuf = torch.empty(need, dtype=torch.uint8).pin_memory()
        assert lib.asfd_set_workspace(h, ctypes.c_void_p(hostbuf.data_ptr()), need) == 1
        assert b"device memory" in lib.asfd_last_error()
        assert lib.asfd_set_workspace(h, None, 5) == 1
        # the plan still works with its own buffers after the refusals
        out = plan.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
    assert rel(out, oracle.eq7(g, u1, d1)) < 1e-5


def test_learned_training_in_workspace(lib):
    g, u1, d1 = W.make("sinusoid64")
    u1_t = torch.as_tensor(u1, device="cuda")
    with FresnelPlan(g, d1, kernel_width=12) as ref_plan:
        ref = ref_plan.execute(u1_t)
    gc.collect()
    with FresnelPlan(g, d1, kind="learned", workspace=True) as plan:
        tables = lib.asfd_debug_live_buffers()
        lib.asfd_debug_fail_allocations(0)
        try:
            losses = [capi.asfd_learned_train_step(plan.handle, u1_t, ref, 1e-3, plan.shape1,
                                                   plan.shape2) for _ in range(3)]
        finally:
            lib.asfd_debug_fail_allocations(-1)
        assert lib.asfd_debug_live_buffers() == tables
        assert all(np.isfinite(losses))
