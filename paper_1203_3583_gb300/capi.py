"""Python binding of the C ABI in include/asfd.h (ctypes; marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of the method: it checks tensor devices, dtypes and shapes, passes
raw pointers and the current CUDA stream, and turns a non-OK status into an
AsfdError carrying asfd_last_error().  PyTorch supplies device memory and
streams.  There is no CPU fallback: if libasfd.so has not been built, loading
fails with an error.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libasfd.so")

ASFD_OK = 0
ASFD_ERR_ARG = 1
ASFD_ERR_NOMEM = 3
ASFD_KERNEL_ES = 0
ASFD_KERNEL_LEARNED = 1

# every symbol declared in include/asfd.h, with (restype, argtypes)
_vp = ctypes.c_void_p
_int = ctypes.c_int


class AsfdError(RuntimeError):
    """A non-OK asfd_status; `.status` holds the code."""

    def __init__(self, status: int, msg: str):
        super().__init__(msg)
        self.status = status


class Params(ctypes.Structure):
    """Mirror of asfd_params."""

    _fields_ = [
        ("n1x", ctypes.c_int), ("n1y", ctypes.c_int),
        ("p1x", ctypes.c_double), ("p1y", ctypes.c_double),
        ("m2x", ctypes.c_int), ("m2y", ctypes.c_int),
        ("p2x", ctypes.c_double), ("p2y", ctypes.c_double),
        ("lam", ctypes.c_double), ("z0", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("kernel_width", ctypes.c_int),
        ("es_beta", ctypes.c_double),
        ("kind", ctypes.c_int),
        ("deterministic", ctypes.c_int),
        ("incidence_sx", ctypes.c_double), ("incidence_sy", ctypes.c_double),
        ("offset_x", ctypes.c_double), ("offset_y", ctypes.c_double),
    ]


class LineParams(ctypes.Structure):
    """Mirror of asfd_line_params."""

    _fields_ = [
        ("m2", ctypes.c_int), ("p2", ctypes.c_double), ("lam", ctypes.c_double),
        ("z0", ctypes.c_double), ("sigma", ctypes.c_double), ("kernel_width", ctypes.c_int),
        ("es_beta", ctypes.c_double), ("incidence_s", ctypes.c_double),
    ]


class PlanInfo(ctypes.Structure):
    """Mirror of asfd_plan_info."""

    _fields_ = [
        ("nfx", ctypes.c_int), ("nfy", ctypes.c_int),
        ("tile_x", ctypes.c_int), ("tile_y", ctypes.c_int),
        ("band_x0", ctypes.c_int), ("band_x1", ctypes.c_int),
        ("band_y0", ctypes.c_int), ("band_y1", ctypes.c_int),
        ("spread_tiles", ctypes.c_int),
        ("tile_pairs", ctypes.c_longlong),
        ("es_beta", ctypes.c_double),
        ("max_abs_eps", ctypes.c_double),
        ("device_bytes", ctypes.c_size_t),
        ("spread_kind", ctypes.c_int),
        ("stride_x", ctypes.c_int), ("stride_y", ctypes.c_int),
        ("run_rows", ctypes.c_int),
    ]


class BatchInfo(ctypes.Structure):
    """Mirror of asfd_batch_info."""

    _fields_ = [
        ("surfaces", ctypes.c_int), ("blocks", ctypes.c_int), ("threads_per_block", ctypes.c_int),
        ("spread_items", ctypes.c_int), ("row_items", ctypes.c_int), ("col_items", ctypes.c_int),
        ("graph", ctypes.c_int), ("source_samples", ctypes.c_longlong),
        ("schedule", ctypes.c_int), ("persistent_ok", ctypes.c_int), ("streams", ctypes.c_int),
    ]


SIGNATURES = {
    "asfd_batch_create": (_int, [ctypes.POINTER(_vp), ctypes.POINTER(Params),
                                 ctypes.POINTER(_vp), _int, _vp]),
    "asfd_batch_execute": (_int, [_vp, ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp]),
    "asfd_batch_get_info": (_int, [_vp, ctypes.POINTER(BatchInfo)]),
    "asfd_batch_set_schedule": (_int, [_vp, _int]),
    "asfd_batch_destroy": (_int, [_vp]),
    "asfd_plan_create": (_int, [ctypes.POINTER(_vp), ctypes.POINTER(Params), _vp, _vp]),
    "asfd_plan_update_d1": (_int, [_vp, _vp, _vp]),
    "asfd_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(Params)]),
    "asfd_set_workspace": (_int, [_vp, _vp, ctypes.c_size_t]),
    "asfd_execute": (_int, [_vp, _vp, _vp, _vp]),
    "asfd_execute_host": (_int, [_vp, _vp, _vp, _vp]),
    "asfd_execute_host_async": (_int, [_vp, _vp, _vp, _vp]),
    "asfd_execute_stage": (_int, [_vp, _int, _vp, _vp, _vp]),
    "asfd_adjoint": (_int, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "asfd_get_plan_info": (_int, [_vp, ctypes.POINTER(PlanInfo)]),
    "asfd_check_device_status": (_int, [_vp, _vp]),
    "asfd_destroy": (_int, [_vp]),
    "asfd_status_string": (ctypes.c_char_p, [_int]),
    "asfd_last_error": (ctypes.c_char_p, []),
    "asfd_debug_fail_allocations": (None, [_int]),
    "asfd_debug_live_buffers": (ctypes.c_longlong, []),
    "asfd_fft_lines": (_int, [_int, _int, _int, _vp, _vp, _vp]),
    "asfd_direct_sum": (_int, [ctypes.POINTER(Params), _vp, _vp, _int, _int, _vp, _vp, _vp, _vp]),
    "asfd_line_plan_create": (_int, [ctypes.POINTER(_vp), ctypes.POINTER(LineParams), _vp, _vp,
                                     _vp, _int, _vp]),
    "asfd_line_execute": (_int, [_vp, _vp, _vp, _vp]),
    "asfd_line_destroy": (_int, [_vp]),
    "asfd_multi_execute": (_int, [_vp, _vp, _int, _vp, _vp]),
    "asfd_fft_lines_noalloc": (_int, [_int, _int, _int, _vp, _vp, _vp]),
    "asfd_probe_launch": (_int, [_int, _int, _vp, ctypes.c_size_t,
                                 ctypes.POINTER(ctypes.c_double), _vp]),
    "asfd_learned_param_count": (ctypes.c_size_t, []),
    "asfd_learned_get_params": (_int, [_vp, _vp, ctypes.c_size_t]),
    "asfd_learned_set_params": (_int, [_vp, _vp, ctypes.c_size_t, _vp]),
    "asfd_learned_train_step": (_int, [_vp, _vp, _vp, ctypes.c_float,
                                       ctypes.POINTER(ctypes.c_double), _vp]),
    "asfd_learned_gradient": (_int, [_vp, _vp, _vp, _vp, ctypes.c_size_t,
                                     ctypes.POINTER(ctypes.c_double), _vp]),
}


def asfd_fft_lines_noalloc(x: torch.Tensor, sign: int = -1, out: torch.Tensor | None = None,
                           stream=None) -> torch.Tensor:
    """asfd_fft_lines without device allocation inside the library (for
    callers that cannot allocate; the twiddle table is a fixed 128 KiB array
    of the library, shared by all calls on a device)."""
    lines, n = x.shape
    if out is None:
        out = torch.empty_like(x)
    _check(load().asfd_fft_lines_noalloc(n, lines, sign,
                                         _dev_ptr(x, torch.complex64, (lines, n), "x"),
                                         _dev_ptr(out, torch.complex64, (lines, n), "out"),
                                         _stream(stream)))
    return out


PROBES = {"smem_load": 0, "smem_store": 1, "l2_red_v2f32": 2, "ffma2": 3, "mufu_ex2": 4}


def asfd_probe_launch(kind: str, iters: int, scratch: torch.Tensor, stream=None) -> float:
    """Queue one resource probe (include/asfd_peaks.h) on the stream; returns
    the work it queued (bytes, flops or evaluations)."""
    if not (isinstance(scratch, torch.Tensor) and scratch.is_cuda and scratch.is_contiguous()):
        raise TypeError("scratch must be a contiguous CUDA tensor")
    work = ctypes.c_double(0.0)
    _check(load().asfd_probe_launch(PROBES[kind], int(iters), ctypes.c_void_p(scratch.data_ptr()),
                                    scratch.numel() * scratch.element_size(), ctypes.byref(work),
                                    _stream(stream)))
    return work.value


def asfd_batch_create(params_list, d1_list, stream=None):
    n = len(params_list)
    arr = (Params * n)(*params_list)
    ptrs = (_vp * n)(*[_dev_ptr(d, torch.float64, (p.n1y, p.n1x), "d1").value
                       for p, d in zip(params_list, d1_list)])
    out = ctypes.c_void_p()
    _check(load().asfd_batch_create(ctypes.byref(out), arr, ptrs, n, _stream(stream)))
    return out


def asfd_batch_execute(batch, u1_list, u2_list, stream=None) -> None:
    n = len(u1_list)
    for t in list(u1_list) + list(u2_list):
        if not (t.is_cuda and t.dtype == torch.complex64 and t.is_contiguous()):
            raise TypeError("batch fields must be contiguous complex64 CUDA tensors")
    p1 = (_vp * n)(*[t.data_ptr() for t in u1_list])
    p2 = (_vp * n)(*[t.data_ptr() for t in u2_list])
    _check(load().asfd_batch_execute(batch, p1, p2, _stream(stream)))


BATCH_SCHEDULES = {"streams": 0, "persistent": 1}


def asfd_batch_set_schedule(batch, schedule: str) -> None:
    _check(load().asfd_batch_set_schedule(batch, BATCH_SCHEDULES[schedule]))


def asfd_batch_get_info(batch) -> dict:
    info = BatchInfo()
    _check(load().asfd_batch_get_info(batch, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in BatchInfo._fields_}


def asfd_batch_destroy(batch) -> None:
    _check(load().asfd_batch_destroy(batch))


def asfd_learned_gradient(plan, u1, ref, shape1, shape2, stream=None):
    """(gradient as a float32 numpy vector, loss) of the learned model."""
    import numpy as np
    n = asfd_learned_param_count()
    out = np.empty(n, np.float32)
    loss = ctypes.c_double(0.0)
    _check(load().asfd_learned_gradient(plan, _dev_ptr(u1, torch.complex64, shape1, "u1"),
                                        _dev_ptr(ref, torch.complex64, shape2, "ref"),
                                        ctypes.c_void_p(out.ctypes.data), n, ctypes.byref(loss),
                                        _stream(stream)))
    return out, loss.value

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH):
    """Load libasfd.so and declare every entry point (raises if it is missing)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(
                    f"{path} is missing: build it with "
                    "`python -c 'import __graft_entry__ as g; g.build()'` (needs nvcc)")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _check(status: int):
    if status != ASFD_OK:
        lib = load()
        msg = lib.asfd_last_error().decode() or lib.asfd_status_string(status).decode()
        raise AsfdError(status, f"{lib.asfd_status_string(status).decode()}: {msg}")


def _stream(stream):
    if stream is None:
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, torch.cuda.Stream):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _dev_ptr(t: torch.Tensor, dtype, shape, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must have dtype {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def make_params(g: dict, sigma: float = 2.0, kernel_width: int = 7, es_beta: float = 0.0,
                kind: int = ASFD_KERNEL_ES, deterministic: bool = False) -> Params:
    """asfd_params from a geometry dict (keys of workloads.geometry; optional
    sx, sy: direction cosines of the incident plane wave; ox, oy: position of
    the source grid's centre sample)."""
    return Params(int(g["n1x"]), int(g["n1y"]), float(g["p1x"]), float(g["p1y"]),
                  int(g["m2x"]), int(g["m2y"]), float(g["p2x"]), float(g["p2y"]),
                  float(g["lam"]), float(g["z0"]), float(sigma), int(kernel_width),
                  float(es_beta), int(kind), int(bool(deterministic)),
                  float(g.get("sx", 0.0)), float(g.get("sy", 0.0)),
                  float(g.get("ox", 0.0)), float(g.get("oy", 0.0)))


def asfd_plan_create(params: Params, d1: torch.Tensor, stream=None) -> ctypes.c_void_p:
    lib = load()
    ptr = _dev_ptr(d1, torch.float64, (params.n1y, params.n1x), "d1")
    out = ctypes.c_void_p()
    _check(lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(params), ptr, _stream(stream)))
    return out


def asfd_plan_update_d1(plan, d1: torch.Tensor, n1x: int, n1y: int, stream=None) -> None:
    lib = load()
    _check(lib.asfd_plan_update_d1(plan, _dev_ptr(d1, torch.float64, (n1y, n1x), "d1"),
                                   _stream(stream)))


def asfd_workspace_bytes(params: Params) -> int:
    """Bytes of a workspace holding every work buffer of a plan (0 if invalid)."""
    n = int(load().asfd_workspace_bytes(ctypes.byref(params)))
    if n == 0:
        raise AsfdError(ASFD_ERR_ARG, load().asfd_last_error().decode())
    return n


def asfd_set_workspace(plan, ws: torch.Tensor | None) -> None:
    """Hands the plan a caller-owned workspace (a CUDA uint8 tensor of at
    least asfd_workspace_bytes() bytes), or detaches it with ws=None."""
    if ws is None:
        _check(load().asfd_set_workspace(plan, None, 0))
        return
    if not (isinstance(ws, torch.Tensor) and ws.is_cuda and ws.dtype == torch.uint8
            and ws.is_contiguous()):
        raise TypeError("workspace must be a contiguous uint8 CUDA tensor")
    _check(load().asfd_set_workspace(plan, ctypes.c_void_p(ws.data_ptr()), ws.numel()))


def asfd_execute(plan, u1: torch.Tensor, u2: torch.Tensor, shape1, shape2, stream=None) -> None:
    lib = load()
    _check(lib.asfd_execute(plan, _dev_ptr(u1, torch.complex64, shape1, "u1"),
                            _dev_ptr(u2, torch.complex64, shape2, "u2"), _stream(stream)))


def asfd_execute_stage(plan, stage: int, u1, u2, shape1, shape2, stream=None) -> None:
    lib = load()
    p1 = _dev_ptr(u1, torch.complex64, shape1, "u1") if u1 is not None else None
    p2 = _dev_ptr(u2, torch.complex64, shape2, "u2") if u2 is not None else None
    _check(lib.asfd_execute_stage(plan, int(stage), p1, p2, _stream(stream)))


def asfd_adjoint(plan, u1, grad_u2, grad_u1, grad_d1, shape1, shape2, stream=None) -> None:
    lib = load()
    p_u1 = _dev_ptr(u1, torch.complex64, shape1, "u1") if u1 is not None else None
    p_g2 = _dev_ptr(grad_u2, torch.complex64, shape2, "grad_u2")
    p_g1 = _dev_ptr(grad_u1, torch.complex64, shape1, "grad_u1") if grad_u1 is not None else None
    p_gd = _dev_ptr(grad_d1, torch.float32, shape1, "grad_d1") if grad_d1 is not None else None
    _check(lib.asfd_adjoint(plan, p_u1, p_g2, p_g1, p_gd, _stream(stream)))


def asfd_execute_host(plan, u1: torch.Tensor, u2: torch.Tensor, shape1, shape2, stream=None,
                      sync: bool = True) -> None:
    """sync=False calls asfd_execute_host_async: the host tensors must stay
    alive and untouched until the stream reaches the transform."""
    lib = load()
    for t, name, shape in ((u1, "u1", shape1), (u2, "u2", shape2)):
        if t.is_cuda or t.dtype != torch.complex64 or tuple(t.shape) != tuple(shape) \
                or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous complex64 host tensor of shape {shape}")
    fn = lib.asfd_execute_host if sync else lib.asfd_execute_host_async
    _check(fn(plan, ctypes.c_void_p(u1.data_ptr()), ctypes.c_void_p(u2.data_ptr()),
              _stream(stream)))


def asfd_get_plan_info(plan) -> dict:
    lib = load()
    info = PlanInfo()
    _check(lib.asfd_get_plan_info(plan, ctypes.byref(info)))
    return {name: getattr(info, name) for name, _ in PlanInfo._fields_}


def asfd_check_device_status(plan, stream=None) -> None:
    _check(load().asfd_check_device_status(plan, _stream(stream)))


def asfd_destroy(plan) -> None:
    _check(load().asfd_destroy(plan))


def asfd_direct_sum(params: Params, d1: torch.Tensor, u1: torch.Tensor, form: int,
                    mx: torch.Tensor, my: torch.Tensor, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Direct GPU sum of Eq. 2, 5 or 7 (form) at the destination points (mx, my)."""
    npts = int(mx.numel())
    if my.numel() != npts:
        raise ValueError("mx and my must have the same length")
    if out is None:
        out = torch.empty(npts, dtype=torch.complex64, device=u1.device)
    _check(load().asfd_direct_sum(
        ctypes.byref(params), _dev_ptr(d1, torch.float64, (params.n1y, params.n1x), "d1"),
        _dev_ptr(u1, torch.complex64, (params.n1y, params.n1x), "u1"), int(form), npts,
        _dev_ptr(mx, torch.int32, (npts,), "mx"), _dev_ptr(my, torch.int32, (npts,), "my"),
        _dev_ptr(out, torch.complex64, (npts,), "out"), _stream(stream)))
    return out


def asfd_line_plan_create(params: LineParams, x1: torch.Tensor, d1: torch.Tensor,
                          w: torch.Tensor, stream=None) -> ctypes.c_void_p:
    n = int(x1.numel())
    out = ctypes.c_void_p()
    _check(load().asfd_line_plan_create(
        ctypes.byref(out), ctypes.byref(params), _dev_ptr(x1, torch.float64, (n,), "x1"),
        _dev_ptr(d1, torch.float64, (n,), "d1"), _dev_ptr(w, torch.float64, (n,), "w"), n,
        _stream(stream)))
    return out


def asfd_line_execute(plan, u1: torch.Tensor, u2: torch.Tensor, n: int, m2: int,
                      stream=None) -> None:
    _check(load().asfd_line_execute(plan, _dev_ptr(u1, torch.complex64, (n,), "u1"),
                                    _dev_ptr(u2, torch.complex64, (m2,), "u2"), _stream(stream)))


def asfd_multi_execute(plans, u1_list, shapes1, u2: torch.Tensor, shape2, stream=None) -> None:
    n = len(plans)
    if n < 1 or len(u1_list) != n or len(shapes1) != n:
        raise ValueError("one u1 per plan")
    parr = (ctypes.c_void_p * n)(*[ctypes.c_void_p(p.value if hasattr(p, "value") else p)
                                   for p in plans])
    uarr = (ctypes.c_void_p * n)(*[_dev_ptr(u, torch.complex64, sh, "u1")
                                   for u, sh in zip(u1_list, shapes1)])
    _check(load().asfd_multi_execute(parr, uarr, n, _dev_ptr(u2, torch.complex64, shape2, "u2"),
                                     _stream(stream)))


def asfd_line_destroy(plan) -> None:
    _check(load().asfd_line_destroy(plan))


def asfd_fft_lines(x: torch.Tensor, sign: int = -1, out: torch.Tensor | None = None,
                   stream=None) -> torch.Tensor:
    """Batched FFT of the rows of a 2D complex64 CUDA tensor with the library's kernel."""
    lines, n = x.shape
    if out is None:
        out = torch.empty_like(x)
    _check(load().asfd_fft_lines(n, lines, sign, _dev_ptr(x, torch.complex64, (lines, n), "x"),
                                 _dev_ptr(out, torch.complex64, (lines, n), "out"),
                                 _stream(stream)))
    return out


def asfd_learned_param_count() -> int:
    return int(load().asfd_learned_param_count())


def asfd_learned_get_params(plan):
    import numpy as np
    n = asfd_learned_param_count()
    out = np.empty(n, np.float32)
    _check(load().asfd_learned_get_params(plan, ctypes.c_void_p(out.ctypes.data), n))
    return out


def asfd_learned_set_params(plan, params, stream=None) -> None:
    import numpy as np
    p = np.ascontiguousarray(params, np.float32)
    _check(load().asfd_learned_set_params(plan, ctypes.c_void_p(p.ctypes.data), p.size,
                                          _stream(stream)))


def asfd_learned_train_step(plan, u1, ref, lr, shape1, shape2, want_loss=True, stream=None):
    loss = ctypes.c_double(0.0)
    _check(load().asfd_learned_train_step(plan, _dev_ptr(u1, torch.complex64, shape1, "u1"),
                                          _dev_ptr(ref, torch.complex64, shape2, "ref"),
                                          ctypes.c_float(lr),
                                          ctypes.byref(loss) if want_loss else None,
                                          _stream(stream)))
    return loss.value if want_loss else None
