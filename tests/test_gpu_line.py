"""The 1D form with explicit source samples (asfd_line_*) against the 1D FP64
oracle: the paper's two line sources (tilted facets, quadratic curve, with
the layout readings of workloads.line_facets / line_quadratic), random
non-uniform samples in arbitrary order, tilted incidence, kernel widths."""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import line as oline  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import LinePlan  # noqa: E402

pytestmark = pytest.mark.gpu
TOL_ES = 1e-5


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


def run(line, x1, d1, w, u1, **kw):
    with LinePlan(line, x1, d1, w, **kw) as p:
        out = p.execute(torch.as_tensor(u1.astype(np.complex64), device="cuda"))
        torch.cuda.synchronize()
        return out.cpu().numpy()


@pytest.mark.parametrize("shape", ["facets", "quadratic"])
def test_paper_line_sources_match_oracle(shape):
    x1, d1, w = W.line_facets() if shape == "facets" else W.line_quadratic()
    line = W.line_geometry()
    u1 = np.ones(x1.size, np.complex128)
    got = run(line, x1, d1, w, u1)
    ref = oline.line(line, x1, d1, w, u1, 7)
    assert rel_l2(got, ref) < TOL_ES, shape


@pytest.mark.parametrize("s", [0.0, 0.004])
def test_random_nonuniform_samples_any_order(s):
    rng = np.random.default_rng(51)
    n = 3000
    x1 = rng.uniform(-2e-3, 2e-3, n)          # unsorted, uneven, some near-coincident
    d1 = 40e-6 * np.sin(x1 / 3e-4) + rng.uniform(-5e-6, 5e-6, n)
    w = rng.uniform(0.5, 1.5, n) * 4e-3 / n
    u1 = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    line = W.line_geometry(m2=512, p2=8e-6, lam=532e-9, z0=0.3, s=s)
    got = run(line, x1, d1, w, u1)
    ref = oline.line(line, x1, d1, w, u1, 7)
    assert rel_l2(got, ref) < TOL_ES, s


@pytest.mark.parametrize("width", [4, 5, 6, 8, 10])
def test_line_kernel_width_accuracy(width):
    x1, d1, w = W.line_facets()
    line = W.line_geometry()
    u1 = np.exp(1j * np.linspace(0, 30, x1.size))
    got = run(line, x1, d1, w, u1, kernel_width=width)
    ref = oline.line(line, x1, d1, w, u1, 7)
    assert rel_l2(got, ref) < max(5e-6, 3.0 * 10.0 ** (-(width - 1))), width


def test_line_rejects_height_at_z0():
    x1 = np.linspace(-1e-4, 1e-4, 16)
    d1 = np.zeros(16)
    d1[3] = 1.0
    with pytest.raises(capi.AsfdError):
        LinePlan(W.line_geometry(), x1, d1, np.full(16, 1e-5))
