"""The C-ABI library builds, loads and exports every entry point of include/asfd.h.

CPU only: nothing here launches device work.
"""
from __future__ import annotations

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in sorted(os.listdir(os.path.join(ROOT, "include")))
           if f.endswith(".h")]


def declared_entry_points():
    names = set()
    for h in HEADERS:
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(asfd_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    from paper_1203_3583_gb300 import _build
    return _build.build()


def test_header_declares_entry_points():
    names = declared_entry_points()
    assert "asfd_plan_create" in names and "asfd_execute" in names and "asfd_destroy" in names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (asfd_[a-z0-9_]+)\b", out))
    missing = [n for n in declared_entry_points() if n not in exported]
    assert not missing, f"declared but not exported: {missing}"


def test_binding_covers_every_symbol(lib_path):
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    for name in declared_entry_points():
        assert name in capi.SIGNATURES, f"{name} has no binding"
        assert hasattr(lib, name)


def test_status_strings_without_gpu(lib_path):
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    assert lib.asfd_status_string(0) == b"ok"
    assert lib.asfd_status_string(1) == b"invalid argument"
    assert lib.asfd_status_string(99) == b"unknown status"


def test_invalid_arguments_rejected_on_host(lib_path):
    """Validation happens before any device call, so it runs without a GPU."""
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    out = ctypes.c_void_p()
    g = dict(n1x=64, n1y=64, p1x=1e-5, p1y=1e-5, m2x=64, m2y=64, p2x=1e-5, p2y=1e-5,
             lam=633e-9, z0=0.05)
    bad = [
        dict(g, n1x=63),                     # odd size
        dict(g, m2x=0),                      # empty
        dict(g, lam=float("nan")),           # non-finite
        dict(g, z0=-1.0),                    # negative distance
    ]
    for b in bad:
        p = capi.make_params(b)
        rc = lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(p), ctypes.c_void_p(1), None)
        assert rc == 1, (b, rc)
        assert out.value is None
    # sigma * m2 not a power of two -> unsupported
    p = capi.make_params(dict(g, m2x=48))
    assert lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(p), ctypes.c_void_p(1), None) == 5
    p = capi.make_params(g, kernel_width=17)
    assert lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(p), ctypes.c_void_p(1), None) == 5
    # NULL d1
    p = capi.make_params(g)
    assert lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(p), None, None) == 1
    assert b"NULL" in lib.asfd_last_error()


def test_debug_hooks_without_gpu(lib_path):
    """The allocation hook and the live-buffer count touch no device."""
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    assert lib.asfd_debug_live_buffers() >= 0
    lib.asfd_debug_fail_allocations(2)
    lib.asfd_debug_fail_allocations(-1)


def _status(lib, p):
    import ctypes
    out = ctypes.c_void_p()
    rc = lib.asfd_plan_create(ctypes.byref(out), ctypes.byref(p), ctypes.c_void_p(1), None)
    assert out.value is None
    return rc


def test_plan_parameter_checks_without_gpu(lib_path):
    """Every asfd_params field with a rule is checked on the host, before any
    device call, with ASFD_ERR_ARG (1) or ASFD_ERR_UNSUPPORTED (5)."""
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    g = dict(n1x=64, n1y=64, p1x=1e-5, p1y=1e-5, m2x=64, m2y=64, p2x=1e-5, p2y=1e-5,
             lam=633e-9, z0=0.05)
    cases = [
        (capi.make_params(g, kernel_width=1), 5),
        (capi.make_params(g, kind=7), 1),
        (capi.make_params(g, kind=capi.ASFD_KERNEL_LEARNED, kernel_width=7), 5),
        (capi.make_params(g, sigma=1.0), 5),
        (capi.make_params(g, sigma=float("nan")), 1),
        (capi.make_params(g, es_beta=-1.0), 1),
        (capi.make_params(dict(g, sx=0.8, sy=0.7)), 1),          # grazing: sx^2 + sy^2 >= 1
        (capi.make_params(dict(g, sx=float("nan"))), 1),
        (capi.make_params(dict(g, ox=float("inf"))), 1),
        (capi.make_params(dict(g, p2y=0.0)), 1),
        (capi.make_params(dict(g, n1y=70000)), 1),
        (capi.make_params(dict(g, m2x=16384)), 5),               # sigma * m2 above 16384
    ]
    for p, want in cases:
        assert _status(lib, p) == want, (p, want, lib.asfd_last_error())
    p = capi.make_params(g)
    p.deterministic = 2
    assert _status(lib, p) == 1


def test_line_plan_parameter_checks_without_gpu(lib_path):
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    fake = ctypes.c_void_p(1)

    def status(**kw):
        base = dict(m2=1024, p2=1e-5, lam=633e-9, z0=1.0, sigma=2.0, kernel_width=7, es_beta=0.0,
                    incidence_s=0.0)
        base.update(kw)
        p = capi.LineParams(**base)
        out = ctypes.c_void_p()
        rc = lib.asfd_line_plan_create(ctypes.byref(out), ctypes.byref(p), fake, fake, fake, 16, None)
        assert out.value is None
        return rc

    assert status(m2=1023) == 1
    assert status(p2=-1e-5) == 1
    assert status(z0=float("inf")) == 1
    assert status(incidence_s=1.0) == 1
    assert status(kernel_width=1) == 5
    assert status(sigma=1.5) == 5          # 1536 is not a power of two
    assert status(es_beta=-2.0) == 1
    out = ctypes.c_void_p()
    p = capi.LineParams(1024, 1e-5, 633e-9, 1.0, 2.0, 7, 0.0, 0.0)
    assert lib.asfd_line_plan_create(ctypes.byref(out), ctypes.byref(p), fake, fake, fake, 0,
                                     None) == 1  # no samples


def test_direct_sum_checks_without_gpu(lib_path):
    """With no destination points the direct sum validates and returns without
    touching the device."""
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    g = dict(n1x=64, n1y=64, p1x=1e-5, p1y=1e-5, m2x=64, m2y=64, p2x=1e-5, p2y=1e-5,
             lam=633e-9, z0=0.05)
    fake = ctypes.c_void_p(1)

    def status(geom, form=7):
        p = capi.make_params(geom)
        return lib.asfd_direct_sum(ctypes.byref(p), fake, fake, form, 0, None, None, None, None)

    assert status(g) == 0
    assert status(g, form=4) == 1
    assert status(dict(g, n1x=63)) == 1
    assert status(dict(g, lam=0.0)) == 1
    assert status(dict(g, sx=0.6, sy=0.9)) == 1
    assert status(dict(g, oy=float("nan"))) == 1


def test_batch_multi_and_fft_checks_without_gpu(lib_path):
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    g = dict(n1x=64, n1y=64, p1x=1e-5, p1y=1e-5, m2x=64, m2y=64, p2x=1e-5, p2y=1e-5,
             lam=633e-9, z0=0.05)
    fake = ctypes.c_void_p(1)

    def batch(params, count=None):
        arr = (capi.Params * len(params))(*params)
        d1s = (ctypes.c_void_p * len(params))(*([fake] * len(params)))
        out = ctypes.c_void_p()
        rc = lib.asfd_batch_create(ctypes.byref(out), arr, d1s,
                                   len(params) if count is None else count, None)
        assert out.value is None
        return rc

    p7 = capi.make_params(g)
    assert batch([p7], count=0) == 1
    assert batch([capi.make_params(g, kind=capi.ASFD_KERNEL_LEARNED, kernel_width=4)]) == 5
    arr = (capi.Params * 2)(p7, p7)
    d1s = (ctypes.c_void_p * 2)(fake, None)
    out = ctypes.c_void_p()
    assert lib.asfd_batch_create(ctypes.byref(out), arr, d1s, 2, None) == 1  # NULL d1
    assert out.value is None
    # (mixed widths, widths outside 4..8 and fine grids above 4096 are valid
    # batches: only the persistent schedule is then unavailable)
    assert lib.asfd_batch_set_schedule(None, 0) == 1
    # multi-surface sums: empty or NULL inputs
    plans = (ctypes.c_void_p * 1)(None)
    u1s = (ctypes.c_void_p * 1)(fake)
    assert lib.asfd_multi_execute(plans, u1s, 1, fake, None) == 1
    assert lib.asfd_multi_execute(plans, u1s, 0, fake, None) == 1
    # FFT lines: length, sign and buffers
    assert lib.asfd_fft_lines(100, 1, -1, fake, fake, None) == 1
    assert lib.asfd_fft_lines(32768, 1, -1, fake, fake, None) == 1
    assert lib.asfd_fft_lines(64, 1, 0, fake, fake, None) == 1
    assert lib.asfd_fft_lines(64, 1, -1, None, fake, None) == 1
    assert lib.asfd_fft_lines(64, -1, -1, fake, fake, None) == 1


def test_workspace_bytes_without_gpu(lib_path):
    """asfd_workspace_bytes touches no device: its value is the sum of the
    work buffers' sizes (fine grid sigma m2x x sigma m2y, row buffer
    sigma m2y x m2x rounded up to a multiple of 4, staging n1x n1y + m2x m2y, plus 2 m2x m2y for learned
    plans; complex64, each rounded up to 256 bytes), and 0 for invalid
    parameters."""
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    up = lambda b: (b + 255) // 256 * 256  # noqa: E731
    g = dict(n1x=2048, n1y=1000, p1x=4e-6, p1y=4e-6, m2x=1024, m2y=512, p2x=4e-6, p2y=4e-6,
             lam=633e-9, z0=0.1)
    p = capi.make_params(g)
    nfx, nfy = 2048, 1024
    want = up(8 * nfx * nfy) + up(8 * nfy * 1024) + up(8 * 2048 * 1000) + up(8 * 1024 * 512)
    assert lib.asfd_workspace_bytes(p) == want
    pl = capi.make_params(g, kernel_width=4, kind=capi.ASFD_KERNEL_LEARNED)
    assert lib.asfd_workspace_bytes(pl) == want + 2 * up(8 * 1024 * 512)
    # ragged sizes: every region still starts on a 256-byte boundary
    g2 = dict(g, n1x=34, n1y=18, m2x=32, m2y=32)
    assert lib.asfd_workspace_bytes(capi.make_params(g2)) == (
        up(8 * 64 * 64) + up(8 * 64 * 32) + up(8 * 34 * 18) + up(8 * 32 * 32))
    # the row buffer's width is m2x rounded up to the row pass's column groups of 4
    g3 = dict(g, n1x=34, n1y=18, m2x=50, m2y=50)
    assert lib.asfd_workspace_bytes(capi.make_params(g3, sigma=1.28)) == (
        up(8 * 64 * 64) + up(8 * 64 * 52) + up(8 * 34 * 18) + up(8 * 50 * 50))
    assert lib.asfd_workspace_bytes(capi.make_params(dict(g, n1x=63))) == 0
    assert b"even" in lib.asfd_last_error()
    assert lib.asfd_workspace_bytes(None) == 0
    assert lib.asfd_set_workspace(None, None, 0) == 1


def test_probe_argument_checks_without_gpu(lib_path):
    """The resource probes check their arguments before any device call."""
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    work = ctypes.c_double(-1.0)
    fake = ctypes.c_void_p(256)
    assert lib.asfd_probe_launch(capi.PROBES["ffma2"], 1, fake, 0, None, None) == 1
    assert lib.asfd_probe_launch(capi.PROBES["ffma2"], 1, None, 1024, ctypes.byref(work), None) == 1
    assert lib.asfd_probe_launch(capi.PROBES["ffma2"], 0, fake, 1024, ctypes.byref(work), None) == 1
    assert lib.asfd_probe_launch(capi.PROBES["ffma2"], (1 << 20) + 1, fake, 1024,
                                 ctypes.byref(work), None) == 1
    assert lib.asfd_probe_launch(99, 1, fake, 1024, ctypes.byref(work), None) == 1
    assert b"unknown probe" in lib.asfd_last_error()
    assert work.value == -1.0


def test_host_execute_checks_without_gpu(lib_path):
    """NULL plans and buffers are refused before any device call."""
    import ctypes
    from paper_1203_3583_gb300 import capi
    lib = capi.load(lib_path)
    fake = ctypes.c_void_p(256)
    for fn in (lib.asfd_execute_host, lib.asfd_execute_host_async):
        assert fn(None, fake, fake, None) == 1
        assert fn(fake, None, fake, None) == 1
        assert fn(fake, fake, None, None) == 1
