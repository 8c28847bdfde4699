"""High-level handle over the C ABI: one plan per (geometry, height map).

    plan = FresnelPlan(geometry, d1)      # d1: float64 [n1y, n1x] (CUDA tensor or array)
    u2 = plan.execute(u1)                 # u1: complex64 [n1y, n1x] CUDA tensor
    plan.close()

All computation happens in libasfd.so on the current CUDA stream; this class
only owns the plan handle and allocates output tensors through PyTorch.
"""
from __future__ import annotations

import numpy as np
import torch

from . import capi


def _as_cuda_f64(d1) -> torch.Tensor:
    if isinstance(d1, torch.Tensor):
        t = d1.to(device="cuda", dtype=torch.float64)
    else:
        t = torch.as_tensor(np.ascontiguousarray(d1, np.float64), device="cuda")
    return t.contiguous()


class FresnelPlan:
    """Plan for Eq. 8 of the paper on one GPU (see include/asfd.h)."""

    def __init__(self, geometry: dict, d1, sigma: float = 2.0, kernel_width: int = 7,
                 es_beta: float = 0.0, stream=None, kind: str = "es",
                 deterministic: bool = False, workspace: bool = False):
        """workspace=True: the plan's work buffers (fine grid, row buffer,
        host-execute staging, learned training buffers) come from one uint8
        tensor of PyTorch's caching allocator (asfd_set_workspace), so the
        library allocates only the plan's tables."""
        self.geometry = dict(geometry)
        if kind not in ("es", "learned"):
            raise ValueError("kind must be 'es' or 'learned'")
        self.kind = kind
        if kind == "learned":
            kernel_width = 4
        self.params = capi.make_params(
            geometry, sigma=sigma, kernel_width=kernel_width, es_beta=es_beta,
            kind=capi.ASFD_KERNEL_LEARNED if kind == "learned" else capi.ASFD_KERNEL_ES,
            deterministic=deterministic)
        self.shape1 = (int(geometry["n1y"]), int(geometry["n1x"]))
        self.shape2 = (int(geometry["m2y"]), int(geometry["m2x"]))
        self._handle = None
        self.workspace = None
        self._handle = capi.asfd_plan_create(self.params, _as_cuda_f64(d1), stream)
        if workspace:
            self.set_workspace(torch.empty(capi.asfd_workspace_bytes(self.params),
                                           dtype=torch.uint8, device="cuda"))

    def set_workspace(self, ws: torch.Tensor | None) -> None:
        """Attach a caller-owned workspace (uint8 CUDA tensor; kept alive by
        this object) or detach it (None)."""
        capi.asfd_set_workspace(self.handle, ws)
        self.workspace = ws

    @property
    def handle(self):
        if self._handle is None:
            raise RuntimeError("plan is closed")
        return self._handle

    def update_d1(self, d1, stream=None) -> None:
        capi.asfd_plan_update_d1(self.handle, _as_cuda_f64(d1), self.shape1[1], self.shape1[0],
                                 stream)

    def execute(self, u1: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.shape2, dtype=torch.complex64, device=u1.device)
        capi.asfd_execute(self.handle, u1, out, self.shape1, self.shape2, stream)
        return out

    def execute_stage(self, stage: int, u1=None, out=None, stream=None) -> None:
        capi.asfd_execute_stage(self.handle, stage, u1, out, self.shape1, self.shape2, stream)

    def adjoint(self, u1, grad_u2: torch.Tensor, grad_u1=None, grad_d1=None, stream=None):
        """Type-2 adjoint: fills grad_u1 (complex64) and/or grad_d1 (float32)."""
        capi.asfd_adjoint(self.handle, u1, grad_u2, grad_u1, grad_d1, self.shape1, self.shape2,
                          stream)
        return grad_u1, grad_d1

    def __call__(self, u1: torch.Tensor, d1: torch.Tensor | None = None) -> torch.Tensor:
        """Differentiable forward transform.  If d1 is given, the plan is
        rebuilt for it first and gradients flow to it; gradients always flow
        to u1.  The plan must not be updated between forward and backward."""
        if d1 is not None:
            self.update_d1(d1.detach())
            return FresnelFunction.apply(u1, d1, self)
        return FresnelFunction.apply(u1, None, self)

    def execute_host(self, u1: torch.Tensor, out: torch.Tensor, stream=None,
                     sync: bool = True) -> torch.Tensor:
        """Transform host tensors (page-locked ones are read and written over
        the host link while the kernels run).  sync=False only queues the
        work on `stream`: keep u1 and out untouched until it completes."""
        capi.asfd_execute_host(self.handle, u1, out, self.shape1, self.shape2, stream, sync)
        return out

    def info(self) -> dict:
        return capi.asfd_get_plan_info(self.handle)

    def check_device_status(self, stream=None) -> None:
        capi.asfd_check_device_status(self.handle, stream)

    def close(self) -> None:
        if self._handle is not None:
            capi.asfd_destroy(self._handle)
            self._handle = None
        self.workspace = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FresnelBatch:
    """Many surfaces per call (see asfd_batch_create): schedule "streams"
    (the default: each surface's kernels on one of the batch's streams) or
    "persistent" (one cooperative kernel over the whole batch)."""

    def __init__(self, items, kernel_width: int = 7, sigma: float = 2.0, stream=None,
                 deterministic: bool = False):
        """items: list of (geometry, d1)."""
        self.shapes1 = [(int(g["n1y"]), int(g["n1x"])) for g, _ in items]
        self.shapes2 = [(int(g["m2y"]), int(g["m2x"])) for g, _ in items]
        params = [capi.make_params(g, sigma=sigma, kernel_width=kernel_width,
                                   deterministic=deterministic) for g, _ in items]
        d1s = [_as_cuda_f64(d1) for _, d1 in items]
        self._handle = None
        self._handle = capi.asfd_batch_create(params, d1s, stream)

    def execute(self, u1_list, out=None, stream=None):
        if out is None:
            out = [torch.empty(s, dtype=torch.complex64, device="cuda") for s in self.shapes2]
        capi.asfd_batch_execute(self._handle, u1_list, out, stream)
        return out

    def set_schedule(self, schedule: str) -> None:
        capi.asfd_batch_set_schedule(self._handle, schedule)

    def info(self) -> dict:
        return capi.asfd_batch_get_info(self._handle)

    def close(self) -> None:
        if self._handle is not None:
            capi.asfd_batch_destroy(self._handle)
            self._handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class FresnelFunction(torch.autograd.Function):
    """u2 = forward(u1; d1) with the type-2 adjoint as its backward.

    PyTorch's complex-gradient convention (dL/dRe + i dL/dIm for a real loss)
    is the one asfd_adjoint uses, so gradients pass through unchanged; the
    d1 gradient is computed in FP32 and returned in d1's dtype."""

    @staticmethod
    def forward(ctx, u1, d1, plan):
        u1c = u1.contiguous()
        u2 = plan.execute(u1c)
        ctx.plan = plan
        ctx.has_d1 = d1 is not None
        ctx.d1_dtype = d1.dtype if d1 is not None else None
        ctx.save_for_backward(u1c)
        return u2

    @staticmethod
    def backward(ctx, grad_u2):
        (u1,) = ctx.saved_tensors
        plan = ctx.plan
        need_u1 = ctx.needs_input_grad[0]
        need_d1 = ctx.has_d1 and ctx.needs_input_grad[1]
        g2 = grad_u2.contiguous().to(torch.complex64)
        gu1 = torch.empty_like(u1) if need_u1 else None
        gd1 = torch.empty(plan.shape1, dtype=torch.float32, device=u1.device) if need_d1 else None
        if need_u1 or need_d1:
            plan.adjoint(u1 if need_d1 else None, g2, gu1, gd1)
        return gu1, (gd1.to(ctx.d1_dtype) if need_d1 else None), None


def direct_sum(geometry: dict, d1, u1: torch.Tensor, form: int, points, stream=None) -> torch.Tensor:
    """Direct GPU evaluation of Eq. 2, 5 or 7 (`form`) at destination points
    (mx, my) (integer arrays or tensors); returns complex64 values.  A reference
    on sampled points and a measure of the paper's approximations (Eqs. 4, 6)."""
    mx, my = points
    dev = u1.device
    mx_t = torch.as_tensor(mx, dtype=torch.int32, device=dev).contiguous()
    my_t = torch.as_tensor(my, dtype=torch.int32, device=dev).contiguous()
    params = capi.make_params(geometry)
    return capi.asfd_direct_sum(params, _as_cuda_f64(d1), u1, form, mx_t, my_t, stream=stream)


class LinePlan:
    """One-dimensional form with explicit source samples (x1, d1, w): Eq. 7 on
    a line source sampled at arbitrary positions (e.g. along the arc length
    of tilted facets or a curve), evaluated by a 1D NUFFT on the GPU.

    line: dict with m2, p2, lam, z0 and optional s (incidence direction cosine).
    """

    def __init__(self, line: dict, x1, d1, w, sigma: float = 2.0, kernel_width: int = 7,
                 es_beta: float = 0.0, stream=None):
        self.n = int(np.asarray(x1).size)
        self.m2 = int(line["m2"])
        self.params = capi.LineParams(self.m2, float(line["p2"]), float(line["lam"]),
                                      float(line["z0"]), float(sigma), int(kernel_width),
                                      float(es_beta), float(line.get("s", 0.0)))
        t = [_as_cuda_f64(np.ravel(v)) for v in (x1, d1, w)]
        self._handle = None
        self._handle = capi.asfd_line_plan_create(self.params, *t, stream=stream)

    def execute(self, u1: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.m2, dtype=torch.complex64, device=u1.device)
        capi.asfd_line_execute(self._handle, u1, out, self.n, self.m2, stream)
        return out

    def close(self) -> None:
        if self._handle is not None:
            capi.asfd_line_destroy(self._handle)
            self._handle = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def multi_execute(plans, u1_list, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Sum of several surfaces' fields at one destination (plans sharing the
    destination sampling, light, distance, kernel and source sample area; see
    asfd_multi_execute): one fine grid and one 2D FFT for all of them."""
    p0 = plans[0]
    if out is None:
        out = torch.empty(p0.shape2, dtype=torch.complex64, device=u1_list[0].device)
    capi.asfd_multi_execute([p.handle for p in plans], u1_list, [p.shape1 for p in plans], out,
                            p0.shape2, stream)
    return out
