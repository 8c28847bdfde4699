"""CUDA path against the FP64 oracle (discretised Eq. 7), through the C ABI.

Tolerance: relative L2 error <= 1e-5 for the exponential-of-semicircle kernel
at width 7 and oversampling 2 (the accuracy target of the plain method).
Small cases compare every destination point; the full-size workloads compare
seeded random destination points (the oracle is O(N^2) per point), and the
constant-height case compares the full 1024^2 grid against the separable FP64
form that Eq. 7 takes when d1 is constant.
"""
from __future__ import annotations

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle  # noqa: E402
from paper_1203_3583_gb300 import capi, workloads as W  # noqa: E402
from paper_1203_3583_gb300.fresnel import FresnelPlan  # noqa: E402
from tests.oracle_cache import sampled  # noqa: E402

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


def run_gpu(g, u1, d1, **kw):
    with FresnelPlan(g, d1, **kw) as plan:
        u2 = plan.execute(torch.as_tensor(u1, device="cuda"))
        torch.cuda.synchronize()
        plan.check_device_status()
        return u2.cpu().numpy(), plan.info()


# --- the FFT kernel on its own ------------------------------------------------------

@pytest.mark.parametrize("n", [16, 32, 64, 128, 256, 512, 1024, 2048, 4096, 8192, 16384])
@pytest.mark.parametrize("sign", [-1, 1])
def test_fft_lines_against_numpy(n, sign):
    rng = np.random.default_rng(n + (sign > 0))
    lines = 37
    x = (rng.standard_normal((lines, n)) + 1j * rng.standard_normal((lines, n))).astype(np.complex64)
    y = capi.asfd_fft_lines(torch.as_tensor(x, device="cuda"), sign=sign)
    torch.cuda.synchronize()
    ref = np.fft.fft(x.astype(np.complex128), axis=1) if sign < 0 else \
        np.fft.ifft(x.astype(np.complex128), axis=1) * n
    err = rel_l2(y.cpu().numpy(), ref)
    assert err < 1e-6, f"n={n} sign={sign}: {err:.2e}"


def test_fft_lines_in_place():
    rng = np.random.default_rng(5)
    x = (rng.standard_normal((9, 4096)) + 1j * rng.standard_normal((9, 4096))).astype(np.complex64)
    t = torch.as_tensor(x, device="cuda")
    capi.asfd_fft_lines(t, sign=-1, out=t)
    torch.cuda.synchronize()
    assert rel_l2(t.cpu().numpy(), np.fft.fft(x.astype(np.complex128), axis=1)) < 1e-6


# --- the whole transform -------------------------------------------------------------

def test_sinusoid64_full_grid():
    g, u1, d1 = W.make("sinusoid64")
    out, _ = run_gpu(g, u1, d1)
    ref = oracle.eq7(g, u1, d1)
    err = rel_l2(out, ref)
    assert err < TOL_ES, err


def test_ragged_nonsquare_full_grid():
    """Source sizes not a multiple of the 16-sample binning tile, unequal pitches
    and sizes per axis, destination smaller than source, asymmetric field."""
    rng = np.random.default_rng(21)
    g = W.geometry(50, 38, 10e-6, 7e-6, 64, 32, 12e-6, 9e-6, 532e-9, 0.04)
    u1 = (rng.standard_normal((38, 50)) + 1j * rng.standard_normal((38, 50))).astype(np.complex64)
    d1 = W.surface_smooth_random(g, rng, 4.0, 60e-6) - 30e-6
    out, _ = run_gpu(g, u1, d1)
    err = rel_l2(out, oracle.eq7(g, u1, d1))
    assert err < TOL_ES, err


def test_periodic_wrap_full_grid():
    """Samples whose frequency t exceeds pi: positions wrap around the fine grid
    several times (the sum is 2 pi periodic in t)."""
    rng = np.random.default_rng(22)
    g = W.geometry(64, 64, 20e-6, 20e-6, 64, 64, 20e-6, 20e-6, 633e-9, 0.02)
    u1 = (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))).astype(np.complex64)
    d1 = W.surface_sinusoid(g, 40e-6, 400e-6)
    out, info = run_gpu(g, u1, d1)
    assert info["band_x0"] == 0 and info["band_x1"] == info["nfx"]
    assert info["spread_kind"] == 1  # wrapping footprints take the atomic kernel
    err = rel_l2(out, oracle.eq7(g, u1, d1))
    assert err < TOL_ES, err


def test_folding_surface_uses_atomic_spread():
    """A rough surface whose samples swap order on the fine grid (the map
    n -> g is not monotone): the conflict-free kernel does not apply and the
    shared-memory-atomic kernel must give the same accuracy."""
    rng = np.random.default_rng(24)
    g = W.geometry(64, 64, 10e-6, 10e-6, 64, 64, 10e-6, 10e-6, 633e-9, 0.05)
    u1 = (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))).astype(np.complex64)
    d1 = rng.uniform(-4e-3, 4e-3, (64, 64))
    out, info = run_gpu(g, u1, d1)
    assert info["spread_kind"] == 1
    err = rel_l2(out, oracle.eq7(g, u1, d1))
    assert err < TOL_ES, err


@pytest.mark.parametrize("name", ["sinusoid64", "spherical_cap1024", "smooth_random2048",
                                  "tilt_bump4096"])
@pytest.mark.parametrize("deterministic", [False, True])
def test_standard_workloads_spread_kind(name, deterministic):
    """Monotone maps at ES width 7: register windows flushed with atomic adds
    (kind 3) by default.  With deterministic=True: the per-item shared-memory
    tiles and ordered gather (kind 4) where samples are at least a fine cell
    apart and the items' tiles fit the row buffer they borrow (the 2048^2
    workload), else the conflict-free tiles with register windows (kind 2;
    the 64^2 workload's samples are 0.4 cells apart, the larger-alpha 1024^2
    and 4096^2 workloads' tiles exceed the row buffer)."""
    g, _, d1 = W.make(name)
    with FresnelPlan(g, d1, deterministic=deterministic) as plan:
        info = plan.info()
    if not deterministic:
        assert info["spread_kind"] == 3, info
    elif name == "smooth_random2048":
        assert info["spread_kind"] == 4, info
    else:
        assert info["spread_kind"] in (2, 4), info
        if info["spread_kind"] == 2:
            assert info["stride_x"] >= 1 and info["stride_y"] >= 1


@pytest.mark.parametrize("name", ["spherical_cap1024", "smooth_random2048", "tilt_bump4096"])
def test_run_twice(name):
    """Atomic-free spreading gives bit-identical results run to run; the
    default path's float atomics may only change the last bits."""
    g, u1, d1 = W.make(name)
    u = torch.as_tensor(u1, device="cuda")
    for det in (True, False):
        with FresnelPlan(g, d1, deterministic=det) as plan:
            a = plan.execute(u).cpu().numpy()
            b = plan.execute(u).cpu().numpy()
        if det:
            assert np.array_equal(a, b)
        else:
            assert rel_l2(a, b) < 1e-6


@pytest.mark.parametrize("index", [3, 13, 8, 4])
def test_dense_maps_match_oracle(index):
    """Surfaces of the 24-surface batch whose samples are far denser than the
    fine grid (alpha = 0.035, 0.097, 0.215, 0.386): the dense spreading kernel
    (register windows, atomic flushes) against the oracle on sampled points."""
    g, u1, d1 = W.make_batch()[index]
    pts = W.sample_points(g, 1024, seed=200 + index)
    out, info = run_gpu(g, u1, d1)
    assert info["spread_kind"] == 3, info
    ref = oracle.eq7(g, u1, d1, points=pts)
    err = rel_l2(out[pts[1], pts[0]], ref)
    assert err < TOL_ES, (index, err)


@pytest.mark.parametrize("width", [2, 3, 5, 6, 7, 8, 13])
@pytest.mark.parametrize("deterministic", [False, True])
def test_widths_spread_kinds_match_oracle(width, deterministic):
    """Widths up to 7 take the register-window kernels (atomic flushes, or
    atomic-free tiles when deterministic: per-item tiles where they fit the
    row buffer, else conflict-free tiles), wider ones the per-sample
    conflict-free kernel; all against the oracle at the accuracy of the width
    (ES error falls about tenfold per unit of width)."""
    g, u1, d1 = W.make("spherical_cap1024")
    pts = W.sample_points(g, 2048, seed=width)
    out, info = run_gpu(g, u1, d1, kernel_width=width, deterministic=deterministic)
    if width > 7:
        assert info["spread_kind"] == 0, info
    else:
        assert info["spread_kind"] in ((2, 4) if deterministic else (3,)), info
    ref = oracle.eq7(g, u1, d1, points=pts)
    err = rel_l2(out[pts[1], pts[0]], ref)
    assert err < max(5e-6, 3.0 * 10.0 ** (-(width - 1))), (width, err)


@pytest.mark.parametrize("name", ["sinusoid64", "smooth_random2048"])
def test_zero_field_after_nonzero_gives_zero(name):
    """The fine grid is reused between calls: every spreading path must start
    from zero (dense plans clear the band before their atomic adds)."""
    g, u1, d1 = W.make(name)
    with FresnelPlan(g, d1) as plan:
        plan.execute(torch.as_tensor(u1, device="cuda"))
        z = plan.execute(torch.zeros(u1.shape, dtype=torch.complex64, device="cuda"))
        torch.cuda.synchronize()
    assert torch.count_nonzero(z).item() == 0


@pytest.mark.parametrize("name,npts,tilt", [("sinusoid64", None, (0.003, -0.004)),
                                            ("spherical_cap1024", 2048, (0.011, -0.017)),
                                            ("smooth_random2048", 512, (0.011, -0.017))])
@pytest.mark.parametrize("deterministic", [False, True])
def test_tilted_incidence_matches_oracle(name, npts, tilt, deterministic):
    """A plane wave at direction cosines `tilt` instead of normal incidence:
    the linear phase rides in the FP64 axis tables, the depth term
    k d1 (sz - 1) in the per-sample correction.  The tilt keeps the deflected
    beam (z0 s) inside the destination window, where the ES error bound,
    relative to the field's energy, applies."""
    g, u1, d1 = W.make(name)
    g = dict(g, sx=tilt[0], sy=tilt[1])
    u = (u1 * np.exp(1j * (np.arange(u1.size).reshape(u1.shape) % 7))).astype(np.complex64)
    out, _ = run_gpu(g, u, d1, deterministic=deterministic)
    if npts is None:
        err = rel_l2(out, oracle.eq7(g, u, d1))
    else:
        pts = W.sample_points(g, npts, seed=400)
        err = rel_l2(out[pts[1], pts[0]], oracle.eq7(g, u, d1, points=pts))
    assert err < TOL_ES, (name, err)


def test_incidence_rejects_grazing_direction():
    g, u1, d1 = W.make("sinusoid64")
    with pytest.raises(capi.AsfdError):
        FresnelPlan(dict(g, sx=0.8, sy=0.7), d1)


def test_zero_field_gives_zero():
    g, u1, d1 = W.make("sinusoid64")
    out, _ = run_gpu(g, np.zeros_like(u1), d1)
    assert np.all(out == 0)


def test_single_sample():
    g, _, d1 = W.make("sinusoid64")
    u1 = np.zeros((64, 64), np.complex64)
    u1[17, 40] = 0.5 - 0.25j
    out, _ = run_gpu(g, u1, d1)
    assert rel_l2(out, oracle.eq7(g, u1, d1)) < TOL_ES


@pytest.mark.parametrize("width", [4, 5, 6, 7, 8, 10, 12])
def test_kernel_width_accuracy(width):
    """ES error falls roughly tenfold per unit of width until FP32 rounding."""
    g, u1, d1 = W.make("sinusoid64")
    rng = np.random.default_rng(23)
    u1 = (rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64))).astype(np.complex64)
    out, _ = run_gpu(g, u1, d1, kernel_width=width)
    err = rel_l2(out, oracle.eq7(g, u1, d1))
    bound = max(3.0 * 10.0 ** (-(width - 1)), 5e-6)  # FP32 rounding floor ~2e-6
    assert err < bound, (width, err)


def test_spherical_cap1024_sampled():
    g, u1, d1 = W.make("spherical_cap1024")
    pts = W.sample_points(g, 4096, seed=102)
    out, _ = run_gpu(g, u1, d1)
    ref = oracle.eq7(g, u1, d1, points=pts)
    err = rel_l2(out[pts[1], pts[0]], ref)
    assert err < TOL_ES, err


@pytest.mark.parametrize("deterministic", [False, True])
def test_smooth_random2048_sampled(deterministic):
    """4096 seeded destination points of the 2048^2 workload, both spread paths."""
    g, u1, d1, pts, ref = sampled("smooth_random2048", 4096, 103)
    out, _ = run_gpu(g, u1, d1, deterministic=deterministic)
    err = rel_l2(out[pts[1], pts[0]], ref)
    assert err < TOL_ES, err


def test_tilt_bump4096_sampled():
    """4096 seeded destination points of the 4096^2 workload."""
    g, u1, d1, pts, ref = sampled("tilt_bump4096", 4096, 105)
    out, _ = run_gpu(g, u1, d1)
    err = rel_l2(out[pts[1], pts[0]], ref)
    assert err < TOL_ES, err


def _constant_height_reference(g, u1, c):
    """d1 = c: Eq. 7 factorises into Ey (u1 o chirp) Ex^T with 1D FP64 DFT
    matrices at distance r0 = z0 - c, times the destination chirp and the
    global factor (Sec. 2, Eqs. 7-8): an exact full-grid reference."""
    k = 2 * np.pi / g["lam"]
    r0 = g["z0"] - c
    x1 = W.coords(g["n1x"], g["p1x"])
    y1 = W.coords(g["n1y"], g["p1y"])
    x2 = W.coords(g["m2x"], g["p2x"])
    y2 = W.coords(g["m2y"], g["p2y"])
    ex = np.exp(-1j * k * np.outer(x2, x1) / r0)
    ey = np.exp(-1j * k * np.outer(y2, y1) / r0)
    f = u1.astype(np.complex128) * np.outer(np.exp(1j * k * y1 ** 2 / (2 * r0)),
                                            np.exp(1j * k * x1 ** 2 / (2 * r0)))
    s = ey @ f @ ex.T
    outer = np.exp(1j * k * (g["z0"] + (x2[None, :] ** 2 + y2[:, None] ** 2) / (2 * g["z0"]))) / (
        1j * g["lam"] * g["z0"])
    return outer * g["p1x"] * g["p1y"] * s


def test_constant_height_full_grid_2048():
    """The 2048^2 workload's geometry and field on a constant surface: the full
    2048^2 destination grid against the separable FP64 reference."""
    g, u1, _ = W.make("smooth_random2048")
    c = 25e-6
    d1 = np.full((g["n1y"], g["n1x"]), c)
    out, _ = run_gpu(g, u1, d1)
    ref = _constant_height_reference(g, u1, c)
    pts = W.sample_points(g, 16, seed=106)
    assert rel_l2(ref[pts[1], pts[0]], oracle.eq7(g, u1, d1, points=pts)) < 1e-9
    err = rel_l2(out, ref)
    assert err < TOL_ES, err


def test_constant_height_full_grid_1024():
    """d1 = c: Eq. 7 factorises into Ey (u1 o chirp) Ex^T with 1D FP64 DFT
    matrices at distance r0 = z0 - c; compared over the full 1024^2 grid."""
    g, u1, _ = W.make("spherical_cap1024")
    c = 0.4e-3
    d1 = np.full((g["n1y"], g["n1x"]), c)
    out, _ = run_gpu(g, u1, d1)
    ref = _constant_height_reference(g, u1, c)
    # spot-check the separable reference against the oracle itself
    pts = W.sample_points(g, 64, seed=104)
    assert rel_l2(ref[pts[1], pts[0]], oracle.eq7(g, u1, d1, points=pts)) < 1e-9
    err = rel_l2(out, ref)
    assert err < TOL_ES, err


@pytest.mark.parametrize("name", ["sinusoid64", "smooth_random2048"])
@pytest.mark.parametrize("pin_in,pin_out", [(True, True), (False, False), (True, False),
                                            (False, True)])
def test_execute_host_matches_device(name, pin_in, pin_out):
    """Host buffers: page-locked ones are read and written in place by the
    kernels, pageable ones go through the plan's staging copies; both give
    the device-buffer result (the same kernels; only the order of the
    spread's float atomics may differ)."""
    g, u1, d1 = W.make(name)
    with FresnelPlan(g, d1) as plan:
        dev = plan.execute(torch.as_tensor(u1, device="cuda")).cpu().numpy()
        hu1 = torch.as_tensor(u1).clone()
        hu2 = torch.zeros(plan.shape2, dtype=torch.complex64)
        if pin_in:
            hu1 = hu1.pin_memory()
        if pin_out:
            hu2 = hu2.pin_memory()
        for _ in range(2):
            plan.execute_host(hu1, hu2)
            assert rel_l2(hu2.numpy(), dev) < 1e-6


@pytest.mark.parametrize("deterministic", [False, True])
def test_execute_host_async_two_plans_pipeline(deterministic):
    """Queued host-buffer transforms on two plans and two streams, four
    different fields each, all in flight before one synchronisation: every
    output equals the device-buffer transform of its own field."""
    g, u1, d1 = W.make("smooth_random2048")
    rng = np.random.default_rng(77)
    fields = [(u1 * np.exp(1j * rng.uniform(0, 2 * np.pi))).astype(np.complex64)
              for _ in range(8)]
    plans = [FresnelPlan(g, d1, deterministic=deterministic) for _ in range(2)]
    streams = [torch.cuda.Stream() for _ in range(2)]
    try:
        want = [plans[0].execute(torch.as_tensor(f, device="cuda")).cpu().numpy() for f in fields]
        hin = [torch.as_tensor(f).pin_memory() for f in fields]
        hout = [torch.zeros(plans[0].shape2, dtype=torch.complex64).pin_memory() for _ in fields]
        torch.cuda.synchronize()
        for k in range(len(fields)):
            plans[k % 2].execute_host(hin[k], hout[k], stream=streams[k % 2], sync=False)
        torch.cuda.synchronize()
        for k in range(len(fields)):
            err = rel_l2(hout[k].numpy(), want[k])
            assert (err == 0.0) if deterministic else (err < 1e-6), (k, err)
    finally:
        for p in plans:
            p.close()


def test_update_d1_equals_fresh_plan():
    g, u1, d1 = W.make("sinusoid64")
    d1b = -0.5 * d1 + 5e-6
    u1t = torch.as_tensor(u1, device="cuda")
    with FresnelPlan(g, d1) as plan:
        plan.update_d1(d1b)
        a = plan.execute(u1t).cpu().numpy()
    with FresnelPlan(g, d1b) as plan:
        b = plan.execute(u1t).cpu().numpy()
    assert rel_l2(a, b) < 1e-6
    assert rel_l2(a, oracle.eq7(g, u1, d1b)) < TOL_ES


@pytest.mark.parametrize("bad,status", [("nan", 1), ("above_z0", 1), ("too_tall", 5)])
def test_invalid_height_map_rejected(bad, status):
    g, _, d1 = W.make("sinusoid64")
    d1 = d1.copy()
    if bad == "nan":
        d1[3, 4] = np.nan
    elif bad == "above_z0":
        d1[10, 10] = g["z0"] * 1.01
    else:
        d1[10, 10] = 0.2 * g["z0"]
    with pytest.raises(capi.AsfdError) as ei:
        FresnelPlan(g, d1)
    assert ei.value.status == status


@pytest.mark.parametrize("name", ["smooth_random2048", "sinusoid64"])
def test_band_state_across_call_sequences(name):
    """The accumulating spread needs a zero band; the forward row pass clears
    each band cell as it reads it, and the plan clears the band itself only
    when something else wrote it.  Every sequence of calls gives the plain
    forward result: repeated forwards, a spread stage run twice before the
    FFT stages, an adjoint (which writes the grid) before a forward, a height
    map changed and restored, and a different field in between."""
    g, u1, d1 = W.make(name, scale=4 if name == "smooth_random2048" else 1)
    rng = np.random.default_rng(31)
    u1b = (rng.standard_normal(u1.shape) + 1j * rng.standard_normal(u1.shape)).astype(np.complex64)
    with FresnelPlan(g, d1) as plan:
        ut, ub = torch.as_tensor(u1, device="cuda"), torch.as_tensor(u1b, device="cuda")
        ref = plan.execute(ut).cpu().numpy()
        outs = [plan.execute(ut).cpu().numpy()]
        out = torch.empty(plan.shape2, dtype=torch.complex64, device="cuda")
        plan.execute_stage(0, u1=ub)
        plan.execute_stage(0, u1=ut)
        plan.execute_stage(1)
        plan.execute_stage(2, out=out)
        outs.append(out.cpu().numpy())
        gu1 = torch.empty_like(ut)
        plan.adjoint(None, torch.as_tensor(np.conj(ref), device="cuda"), gu1, None)
        outs.append(plan.execute(ut).cpu().numpy())
        plan.update_d1(0.5 * d1)
        plan.execute(ub)
        plan.update_d1(d1)
        outs.append(plan.execute(ut).cpu().numpy())
        plan.execute(ub)
        outs.append(plan.execute(ut).cpu().numpy())
    for i, o in enumerate(outs):
        assert rel_l2(o, ref) < 1e-6, i
    assert rel_l2(ref, oracle.eq7(g, u1, d1) if name == "sinusoid64" else ref) < TOL_ES
