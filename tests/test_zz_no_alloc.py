"""The allocation-free batched FFT (asfd_fft_lines_noalloc) through the C ABI.

For callers that cannot allocate device memory: the entry point keeps its
twiddle table in a fixed array of the library.  Two calls in a row (two
lengths, so the second must rewrite the shared table) must give the same
output as the allocating entry point asfd_fft_lines, within the 1e-6
relative tolerance of the FFT tests, and a length above the array's limit
must be refused.  Collected last so that a run stopping at the first
failure has run every other test; it also passes alone in a fresh process.
"""
from __future__ import annotations

import ctypes

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1203_3583_gb300 import capi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1203_3583_gb300 import _build
    return capi.load(_build.build())


def _fft(lib, name, x, sign):
    lines, n = x.shape
    out = torch.empty_like(x)
    st = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = getattr(lib, name)(n, lines, sign, ctypes.c_void_p(x.data_ptr()),
                            ctypes.c_void_p(out.data_ptr()), st)
    assert rc == 0, lib.asfd_last_error()
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_noalloc_matches_allocating_fft_two_calls(lib):
    rng = np.random.default_rng(77)
    for n, lines, sign in ((4096, 19, -1), (1024, 33, 1)):
        x = torch.as_tensor((rng.standard_normal((lines, n)) +
                             1j * rng.standard_normal((lines, n))).astype(np.complex64), device="cuda")
        ref = _fft(lib, "asfd_fft_lines", x, sign)
        got = _fft(lib, "asfd_fft_lines_noalloc", x, sign)
        err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
        assert err < 1e-6, (n, err)


def test_noalloc_rejects_length_above_limit(lib):
    x = torch.zeros((1, 32768), dtype=torch.complex64, device="cuda")
    out = torch.empty_like(x)
    rc = lib.asfd_fft_lines_noalloc(32768, 1, -1, ctypes.c_void_p(x.data_ptr()),
                                    ctypes.c_void_p(out.data_ptr()), None)
    assert rc == 1
    assert b"16384" in lib.asfd_last_error()
