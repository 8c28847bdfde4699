"""Type-2 adjoint (gradients w.r.t. the source field and the height map).

* the dot-product identity <y, A x> = <A^H y, x> on the GPU pair (exact up to
  FP32 rounding, since the adjoint is the transpose of the discrete forward);
* agreement with the FP64 oracle's gradient of the direct Eq. 7 sum;
* central finite differences of a loss at full size, where each perturbed
  coordinate changes one term of Eq. 7, so the perturbed field is the GPU
  field plus an exact FP64 rank-1 update over all destination points.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan  # noqa: E402

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


def crandn(rng, shape):
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)).astype(np.complex64)


def gpu_adjoint(plan, u1, g):
    gu1 = torch.empty(plan.shape1, dtype=torch.complex64, device="cuda")
    gd1 = torch.empty(plan.shape1, dtype=torch.float32, device="cuda")
    plan.adjoint(torch.as_tensor(u1, device="cuda"), torch.as_tensor(g, device="cuda"), gu1, gd1)
    torch.cuda.synchronize()
    return gu1.cpu().numpy(), gd1.cpu().numpy()


CASES = {
    "sinusoid64": lambda: W.make("sinusoid64"),
    "ragged": lambda: (W.geometry(50, 38, 10e-6, 7e-6, 64, 32, 12e-6, 9e-6, 532e-9, 0.04), None,
                       None),
    # a plane wave incident at direction cosines (0.012, -0.02): its depth
    # term k d1 (sz - 1) adds to the d1 gradient
    "ragged_tilted": lambda: (dict(W.geometry(50, 38, 10e-6, 7e-6, 64, 32, 12e-6, 9e-6, 532e-9,
                                              0.04), sx=0.012, sy=-0.02), None, None),
}


def _case(name, rng):
    g, u1, d1 = CASES[name]()
    if u1 is None:
        u1 = crandn(rng, (g["n1y"], g["n1x"]))
        d1 = W.surface_smooth_random(g, rng, 4.0, 60e-6) - 30e-6
    return g, u1, d1


@pytest.mark.parametrize("name", sorted(CASES))
def test_dot_product_identity(name):
    rng = np.random.default_rng(31)
    g, _, d1 = _case(name, rng)
    x = crandn(rng, (g["n1y"], g["n1x"]))
    y = crandn(rng, (g["m2y"], g["m2x"]))
    with FresnelPlan(g, d1) as plan:
        ax = plan.execute(torch.as_tensor(x, device="cuda")).cpu().numpy()
        ahy, _ = gpu_adjoint(plan, x, y)
    lhs = np.vdot(y.astype(np.complex128), ax.astype(np.complex128))
    rhs = np.vdot(ahy.astype(np.complex128), x.astype(np.complex128))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("name", sorted(CASES))
def test_gradients_match_oracle(name):
    rng = np.random.default_rng(32)
    g, u1, d1 = _case(name, rng)
    u1 = crandn(rng, u1.shape)
    gu2 = crandn(rng, (g["m2y"], g["m2x"]))
    with FresnelPlan(g, d1) as plan:
        gu1, gd1 = gpu_adjoint(plan, u1, gu2)
    ref_u1, ref_d1 = oracle.eq7_grad(g, u1, d1, gu2)
    assert rel_l2(gu1, ref_u1) < 1e-5
    assert rel_l2(gd1, ref_d1) < 1e-4, rel_l2(gd1, ref_d1)


def test_autograd_function_loss():
    """L = sum (|u2|^2 - T)^2 through torch.autograd with the adjoint backward."""
    rng = np.random.default_rng(33)
    g, u1, d1 = W.make("sinusoid64")
    u1 = crandn(rng, u1.shape)
    u1_t = torch.as_tensor(u1, device="cuda").requires_grad_(True)
    d1_t = torch.as_tensor(d1, device="cuda").requires_grad_(True)
    with FresnelPlan(g, d1) as plan:
        u2 = plan(u1_t, d1_t)
        inten = u2.real ** 2 + u2.imag ** 2
        target = torch.rand_like(inten) * 2 * inten.mean().detach()
        loss = ((inten - target) ** 2).sum()
        loss.backward()
    u2n = u2.detach().cpu().numpy().astype(np.complex128)
    gu2 = 4 * (np.abs(u2n) ** 2 - target.cpu().numpy()) * u2n
    ref_u1, ref_d1 = oracle.eq7_grad(g, u1, d1, gu2)
    assert rel_l2(u1_t.grad.cpu().numpy(), ref_u1) < 1e-4
    assert rel_l2(d1_t.grad.cpu().numpy(), ref_d1) < 1e-4


def _rank1_delta(g, u1n, d1n, nx, ny, u_new, h_new, outer):
    """Exact FP64 change of the Eq. 7 field when sample (nx, ny) changes from
    (u1n, d1n) to (u_new, h_new); `outer` = exp(ik(z0+|x2|^2/2z0))/(i lam z0) p1x p1y."""
    k = 2 * np.pi / g["lam"]
    x1 = (nx - g["n1x"] // 2) * g["p1x"]
    y1 = (ny - g["n1y"] // 2) * g["p1y"]
    mxp = np.arange(g["m2x"]) - g["m2x"] // 2
    myp = np.arange(g["m2y"]) - g["m2y"] // 2

    def term(u, h):
        r0 = g["z0"] - h
        ph = k * h + k * (-h + (x1 * x1 + y1 * y1) / (2 * r0))
        ex = np.exp(-1j * k * g["p2x"] * x1 / r0 * mxp)
        ey = np.exp(-1j * k * g["p2y"] * y1 / r0 * myp)
        return u * np.exp(1j * ph) * np.outer(ey, ex)

    return outer * (term(u_new, h_new) - term(u1n, d1n))


def _fd_check(name, ncoord, seed):
    g, u1, d1 = W.make(name) if name != "tilt_bump1024" else W.make("tilt_bump4096", scale=4)
    rng = np.random.default_rng(seed)
    u1_t = torch.as_tensor(u1, device="cuda")
    with FresnelPlan(g, d1) as plan:
        u2_t = plan.execute(u1_t)
        inten = (u2_t.abs() ** 2).double()
        target = torch.rand(inten.shape, generator=torch.Generator().manual_seed(seed),
                            dtype=torch.float64).to("cuda") * 2 * inten.mean()
        gu2 = (4 * (inten - target) * u2_t.to(torch.complex128)).to(torch.complex64)
        gu1 = torch.empty_like(u1_t)
        gd1 = torch.empty(plan.shape1, dtype=torch.float32, device="cuda")
        plan.adjoint(u1_t, gu2, gu1, gd1)
        torch.cuda.synchronize()
    u2 = u2_t.cpu().numpy().astype(np.complex128)
    T = target.cpu().numpy()
    gd1 = gd1.cpu().numpy().astype(np.float64)
    gu1 = gu1.cpu().numpy().astype(np.complex128)
    k = 2 * np.pi / g["lam"]
    x2 = W.coords(g["m2x"], g["p2x"])[None, :]
    y2 = W.coords(g["m2y"], g["p2y"])[:, None]
    outer = (np.exp(1j * k * (g["z0"] + (x2 ** 2 + y2 ** 2) / (2 * g["z0"]))) / (1j * g["lam"] * g["z0"])
             * g["p1x"] * g["p1y"])

    def dloss(dp, dm):
        ip = np.abs(u2 + dp) ** 2
        im = np.abs(u2 + dm) ** 2
        return float(np.sum((ip - im) * (ip + im - 2 * T)))

    flat = rng.choice(g["n1x"] * g["n1y"], size=ncoord, replace=False)
    h = 1e-3 / k                    # ~1e-3 rad of phase
    dphi = 1e-3                     # source phase step
    err_d1, err_ph, scale_d1, scale_ph = [], [], [], []
    for f in flat:
        nx, ny = int(f % g["n1x"]), int(f // g["n1x"])
        un = complex(u1[ny, nx])
        dn = float(d1[ny, nx])
        fd = dloss(_rank1_delta(g, un, dn, nx, ny, un, dn + h, outer),
                   _rank1_delta(g, un, dn, nx, ny, un, dn - h, outer)) / (2 * h)
        err_d1.append(fd - gd1[ny, nx])
        scale_d1.append(fd)
        # source phase: u1 -> u1 exp(+-i dphi); dL/dphi = Re(conj(gu1) i u1)
        fdp = dloss(_rank1_delta(g, un, dn, nx, ny, un * np.exp(1j * dphi), dn, outer),
                    _rank1_delta(g, un, dn, nx, ny, un * np.exp(-1j * dphi), dn, outer)) / (2 * dphi)
        ana = float(np.real(np.conj(gu1[ny, nx]) * 1j * un))
        err_ph.append(fdp - ana)
        scale_ph.append(fdp)
    e1 = np.linalg.norm(err_d1) / np.linalg.norm(scale_d1)
    e2 = np.linalg.norm(err_ph) / np.linalg.norm(scale_ph)
    return e1, e2


def test_finite_differences_tilt_bump1024():
    e_d1, e_ph = _fd_check("tilt_bump1024", 64, 41)
    assert e_d1 < 1e-3, e_d1
    assert e_ph < 1e-3, e_ph


def test_finite_differences_tilt_bump4096():
    """The full-size adjoint workload (4096^2 source at 3.74 um, tilted plane
    plus Gaussian bump, 532 nm, z0 = 0.15 m), 64 seeded coordinates."""
    e_d1, e_ph = _fd_check("tilt_bump4096", 64, 42)
    assert e_d1 < 1e-3, e_d1
    assert e_ph < 1e-3, e_ph
