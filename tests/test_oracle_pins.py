"""The FP64 oracle against references that do not reuse its formula (CPU only).

The forward pins are in tests/oracle_pins.py.  The gradient routine is pinned
to the (already pinned) forward oracle by central finite differences and by
the exact adjoint identity <A x, y> = <x, A^H y>.  The mutation test plants
plausible mistakes in a copy of the oracle's C source (flipped sign, dropped
factor, swapped pitch, shifted origin, z0 for r0 ...) and checks that every
mutant fails at least one pin.
"""
from __future__ import annotations

import os

import numpy as np
import pytest

import oracle
from tests import oracle_pins as pins


@pytest.mark.parametrize("name", sorted(pins.ALL_PINS))
def test_forward_pin(name):
    fn, tol = pins.ALL_PINS[name]
    err = fn(oracle.eq7)
    assert err < tol, f"{name}: rel err {err:.3e} >= {tol:.1e}"


def test_sampled_points_match_full_grid():
    rng = np.random.default_rng(1)
    g = dict(n1x=12, n1y=10, p1x=8e-6, p1y=9e-6, m2x=14, m2y=8, p2x=10e-6, p2y=11e-6,
             lam=532e-9, z0=0.03)
    u1 = rng.standard_normal((10, 12)) + 1j * rng.standard_normal((10, 12))
    d1 = rng.uniform(-1e-4, 1e-4, (10, 12))
    full = oracle.eq7(g, u1, d1)
    mx = np.array([0, 13, 5, 7], np.int32)
    my = np.array([0, 7, 3, 2], np.int32)
    pts = oracle.eq7(g, u1, d1, points=(mx, my))
    np.testing.assert_array_equal(pts, full[my, mx])


def test_linearity_over_sample_subsets():
    rng = np.random.default_rng(2)
    g = dict(n1x=16, n1y=12, p1x=10e-6, p1y=10e-6, m2x=10, m2y=10, p2x=12e-6, p2y=12e-6,
             lam=633e-9, z0=0.05)
    u1 = rng.standard_normal((12, 16)) + 1j * rng.standard_normal((12, 16))
    d1 = rng.uniform(-2e-4, 2e-4, (12, 16))
    mask = rng.random((12, 16)) < 0.4
    whole = oracle.eq7(g, u1, d1)
    parts = oracle.eq7(g, np.where(mask, u1, 0), d1) + oracle.eq7(g, np.where(mask, 0, u1), d1)
    assert pins.rel_l2(parts, whole) < 1e-13


def test_even_source_gives_even_field():
    """Even u1 and even d1 about the grid centre give an even u2 (index n -> N - n)."""
    n = 16
    rng = np.random.default_rng(3)
    a = rng.standard_normal((n + 1, n + 1)) + 1j * rng.standard_normal((n + 1, n + 1))
    a = a + a[::-1, ::-1]
    h = rng.uniform(0, 1e-4, (n + 1, n + 1))
    h = h + h[::-1, ::-1]
    # centred grids of even size: index 0 has no mirror partner; zero it
    u1 = a[:n, :n].copy()
    d1 = h[:n, :n].copy()
    u1[0, :] = 0
    u1[:, 0] = 0
    g = dict(n1x=n, n1y=n, p1x=10e-6, p1y=10e-6, m2x=n, m2y=n, p2x=9e-6, p2y=9e-6,
             lam=633e-9, z0=0.05)
    out = oracle.eq7(g, u1, d1)
    inner = out[1:, 1:]
    np.testing.assert_allclose(inner, inner[::-1, ::-1], rtol=1e-10, atol=1e-10 * np.abs(out).max())


# --- gradient routine ----------------------------------------------------------

def _grad_case(seed=4):
    rng = np.random.default_rng(seed)
    g = dict(n1x=10, n1y=8, p1x=10e-6, p1y=12e-6, m2x=12, m2y=10, p2x=11e-6, p2y=9e-6,
             lam=633e-9, z0=0.04)
    u1 = rng.standard_normal((8, 10)) + 1j * rng.standard_normal((8, 10))
    d1 = rng.uniform(-3e-4, 3e-4, (8, 10))
    target = rng.random((10, 12)) * 2 * np.mean(np.abs(oracle.eq7(g, u1, d1)) ** 2)
    return g, u1, d1, target


def _loss(g, u1, d1, target):
    i = np.abs(oracle.eq7(g, u1, d1)) ** 2
    return float(np.sum((i - target) ** 2))


def _loss_grad_u2(u2, target):
    # L = sum (|u|^2 - T)^2 ; dL/dRe u + i dL/dIm u = 4 (|u|^2 - T) u
    return 4 * (np.abs(u2) ** 2 - target) * u2


def test_grad_d1_central_differences():
    g, u1, d1, target = _grad_case()
    u2 = oracle.eq7(g, u1, d1)
    _, gd1 = oracle.eq7_grad(g, u1, d1, _loss_grad_u2(u2, target))
    h = 2e-10  # k h ~ 2e-3 rad
    for (iy, ix) in [(0, 0), (3, 7), (7, 9), (5, 2)]:
        dp = d1.copy()
        dm = d1.copy()
        dp[iy, ix] += h
        dm[iy, ix] -= h
        fd = (_loss(g, u1, dp, target) - _loss(g, u1, dm, target)) / (2 * h)
        assert abs(fd - gd1[iy, ix]) <= 2e-5 * abs(gd1).max(), (iy, ix, fd, gd1[iy, ix])


def test_grad_u1_central_differences():
    g, u1, d1, target = _grad_case(5)
    u2 = oracle.eq7(g, u1, d1)
    gu1, _ = oracle.eq7_grad(g, u1, d1, _loss_grad_u2(u2, target))
    h = 1e-6
    for (iy, ix) in [(1, 1), (6, 4)]:
        for unit, part in ((1.0, "re"), (1j, "im")):
            up = u1.copy()
            um = u1.copy()
            up[iy, ix] += h * unit
            um[iy, ix] -= h * unit
            fd = (_loss(g, up, d1, target) - _loss(g, um, d1, target)) / (2 * h)
            ana = gu1[iy, ix].real if part == "re" else gu1[iy, ix].imag
            assert abs(fd - ana) <= 1e-6 * np.abs(gu1).max(), (iy, ix, part, fd, ana)


def test_grad_u1_adjoint_identity():
    """<A x, y> = <x, A^H y> with A the (pinned) forward oracle."""
    rng = np.random.default_rng(6)
    g = dict(n1x=14, n1y=10, p1x=10e-6, p1y=8e-6, m2x=12, m2y=16, p2x=9e-6, p2y=13e-6,
             lam=532e-9, z0=0.06)
    x = rng.standard_normal((10, 14)) + 1j * rng.standard_normal((10, 14))
    y = rng.standard_normal((16, 12)) + 1j * rng.standard_normal((16, 12))
    d1 = rng.uniform(-2e-4, 4e-4, (10, 14))
    ax = oracle.eq7(g, x, d1)
    ahy, _ = oracle.eq7_grad(g, x, d1, y)
    lhs = np.vdot(y, ax)
    rhs = np.vdot(ahy, x)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


# --- planted mistakes must fail a pin -------------------------------------------

MUTANTS = {
    "cross_sign": ("const double ph_x = -k * (x1x * x2x", "const double ph_x = k * (x1x * x2x"),
    "drop_incident": ("const double ph = ph_inc + ph_src + ph_x;\n                const double c",
                      "const double ph = ph_src + ph_x;\n                const double c"),
    "chirp_z0_for_r0": ("const double ph_src = k * (-h + (x1x * x1x + x1y * x1y) / (2.0 * r0));\n"
                        "                /* exp(-ik",
                        "const double ph_src = k * (-h + (x1x * x1x + x1y * x1y) / (2.0 * g->z0));\n"
                        "                /* exp(-ik"),
    "cross_z0_for_r0": ("const double ph_x = -k * (x1x * x2x + x1y * x2y) / r0;\n                const double ph =",
                        "const double ph_x = -k * (x1x * x2x + x1y * x2y) / g->z0;\n                const double ph ="),
    "swap_dest_pitch": ("const double x2x = (mx[i] - g->m2x / 2) * g->p2x;\n        const double x2y = (my[i] - g->m2y / 2) * g->p2y;\n        double acc_re",
                        "const double x2x = (mx[i] - g->m2x / 2) * g->p2y;\n        const double x2y = (my[i] - g->m2y / 2) * g->p2x;\n        double acc_re"),
    "source_origin": ("const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;\n                const double h",
                      "const double x1x = (nx - g->n1x / 2 + 1) * g->p1x + g->ox;\n                const double h"),
    "offset_sign": ("const double x1x = (nx - g->n1x / 2) * g->p1x + g->ox;\n                const double h",
                    "const double x1x = (nx - g->n1x / 2) * g->p1x - g->ox;\n                const double h"),
    "drop_dest_chirp": ("const double ph = k * (g->z0 + (x2x * x2x + x2y * x2y) / (2.0 * g->z0));",
                        "const double ph = k * (g->z0);"),
    "conj_accumulate": ("row_im += ur * s + ui * c;", "row_im += ur * s - ui * c;"),
    "prefactor_sign": ("*im = -cos(ph) / a;", "*im = cos(ph) / a;"),
    "drop_weight": ("acc_re *= w;\n        acc_im *= w;", "acc_re *= 1.0;\n        acc_im *= 1.0;"),
    "transpose_index": ("const size_t n = (size_t)ny * g->n1x + nx;",
                        "const size_t n = (size_t)nx * g->n1y + ny;"),
    "tilt_sign": ("return k * (g->sx * x + g->sy * y + sz * h);",
                  "return k * (-g->sx * x + g->sy * y + sz * h);"),
    "tilt_depth_cosine": ("return k * (g->sx * x + g->sy * y + sz * h);",
                          "return k * (g->sx * x + g->sy * y + h);"),
    "tilt_swap_axes": ("return k * (g->sx * x + g->sy * y + sz * h);",
                       "return k * (g->sy * x + g->sx * y + sz * h);"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "asfd_oracle.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) >= 1, f"mutation anchor for {name} not found"
    mutated = src.replace(old, new, 1)
    cpath = tmp_path / "mutant.c"
    cpath.write_text(mutated)
    lib = oracle.bind(oracle.compile_c(str(cpath), str(tmp_path / "libmutant.so")))

    def eq7(g, u1, d1, points=None):
        return oracle.eq7(g, u1, d1, points=points, lib=lib)

    failures = []
    for pname, (fn, tol) in pins.ALL_PINS.items():
        try:
            err = fn(eq7)
        except IndexError:
            err = np.inf
        if not err < tol:
            failures.append(pname)
    assert failures, f"mutant {name} passed every pin"


# --- Eq. 5 and Eq. 2 --------------------------------------------------------------

def _direct_fns(lib=None):
    def eq5(g, u1, d1, points=None):
        return oracle.eq5(g, u1, d1, points=points, lib=lib)

    def eq2(g, u1, d1, points=None):
        return oracle.eq2(g, u1, d1, points=points, lib=lib)

    def eq7(g, u1, d1, points=None):
        return oracle.eq7(g, u1, d1, points=points, lib=lib)
    return eq5, eq2, eq7


@pytest.mark.parametrize("name", sorted(pins.DIRECT_PINS))
def test_direct_pin(name):
    fn, tol = pins.DIRECT_PINS[name]
    err = fn(*_direct_fns())
    assert err < tol, f"{name}: {err:.3e} >= {tol:.1e}"


DIRECT_MUTANTS = {
    "eq5_dest_chirp_z0": ("const double ph_dst = k * x2sq / (2.0 * r0);",
                          "const double ph_dst = k * x2sq / (2.0 * g->z0);"),
    "eq5_drop_dest_chirp": ("const double ph = ph_inc + ph_src + ph_x + ph_dst;",
                            "const double ph = ph_inc + ph_src + ph_x;"),
    "eq5_drop_incident": ("const double ph = ph_inc + ph_src + ph_x + ph_dst;",
                          "const double ph = ph_src + ph_x + ph_dst;"),
    "eq2_distance_z0": ("const double dx = x2x - x1x, dy = x2y - x1y, dz = g->z0 - h;",
                        "const double dx = x2x - x1x, dy = x2y - x1y, dz = g->z0;"),
    "eq2_phase_sign": ("const double ph = incident_phase(g, k, x1x, x1y, h) + k * r;",
                       "const double ph = incident_phase(g, k, x1x, x1y, h) - k * r;"),
    "eq2_drop_incident": ("const double ph = incident_phase(g, k, x1x, x1y, h) + k * r;",
                          "const double ph = k * r;"),
    "eq2_prefactor_sign": ("out[2 * i] = f * acc_im;\n        out[2 * i + 1] = -f * acc_re;",
                           "out[2 * i] = -f * acc_im;\n        out[2 * i + 1] = f * acc_re;"),
}


@pytest.mark.parametrize("name", sorted(DIRECT_MUTANTS))
def test_planted_mistake_in_direct_sums_fails_a_pin(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "asfd_oracle.c")).read()
    old, new = DIRECT_MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(src.replace(old, new, 1))
    lib = oracle.bind(oracle.compile_c(str(cpath), str(tmp_path / "libmutant.so")))
    failures = [p for p, (fn, tol) in pins.DIRECT_PINS.items()
                if not fn(*_direct_fns(lib)) < tol]
    assert failures, f"mutant {name} passed every pin"


# --- planted mistakes in the gradient routine must fail a gradient pin ----------

def _grad_errors(lib=None):
    """Worst relative errors of asfd_oracle_eq7_grad (from `lib`) against central
    differences of the unmodified forward oracle, at normal and tilted incidence,
    and against the adjoint identity."""
    errs = {}
    h = 2e-10
    for name, seed, tilt in (("d1", 4, (0.0, 0.0)), ("d1_tilted", 7, (0.02, -0.015))):
        g, u1, d1, target = _grad_case(seed)
        g = dict(g, sx=tilt[0], sy=tilt[1])
        u2 = oracle.eq7(g, u1, d1)
        _, gd1 = oracle.eq7_grad(g, u1, d1, _loss_grad_u2(u2, target), lib=lib)
        fds, anas = [], []
        for (iy, ix) in [(0, 0), (3, 7), (7, 9), (5, 2)]:
            dp = d1.copy()
            dm = d1.copy()
            dp[iy, ix] += h
            dm[iy, ix] -= h
            fds.append((_loss(g, u1, dp, target) - _loss(g, u1, dm, target)) / (2 * h))
            anas.append(gd1[iy, ix])
        fds, anas = np.array(fds), np.array(anas)
        errs[name] = float(np.max(np.abs(fds - anas)) / np.max(np.abs(fds)))
    g, u1, d1, target = _grad_case(5)
    u2 = oracle.eq7(g, u1, d1)
    gu1, _ = oracle.eq7_grad(g, u1, d1, _loss_grad_u2(u2, target), lib=lib)
    fds, anas = [], []
    for (iy, ix) in [(1, 1), (6, 4)]:
        for unit, part in ((1.0, "re"), (1j, "im")):
            up = u1.copy()
            um = u1.copy()
            up[iy, ix] += 1e-6 * unit
            um[iy, ix] -= 1e-6 * unit
            fds.append((_loss(g, up, d1, target) - _loss(g, um, d1, target)) / 2e-6)
            anas.append(gu1[iy, ix].real if part == "re" else gu1[iy, ix].imag)
    fds, anas = np.array(fds), np.array(anas)
    errs["u1"] = float(np.max(np.abs(fds - anas)) / np.max(np.abs(fds)))
    rng = np.random.default_rng(6)
    g = dict(n1x=14, n1y=10, p1x=10e-6, p1y=8e-6, m2x=12, m2y=16, p2x=9e-6, p2y=13e-6,
             lam=532e-9, z0=0.06)
    x = rng.standard_normal((10, 14)) + 1j * rng.standard_normal((10, 14))
    y = rng.standard_normal((16, 12)) + 1j * rng.standard_normal((16, 12))
    d1 = rng.uniform(-2e-4, 4e-4, (10, 14))
    lhs = np.vdot(y, oracle.eq7(g, x, d1))
    ahy, _ = oracle.eq7_grad(g, x, d1, y, lib=lib)
    errs["adjoint"] = float(abs(lhs - np.vdot(ahy, x)) / abs(lhs))
    return errs


GRAD_TOL = {"d1": 1e-4, "d1_tilted": 1e-4, "u1": 1e-5, "adjoint": 1e-12}


def test_gradient_pins_hold():
    errs = _grad_errors()
    for name, tol in GRAD_TOL.items():
        assert errs[name] < tol, (name, errs[name])


GRAD_MUTANTS = {
    "grad_source_chirp_sign": (
        "const double dph_common = k * sz - k + k * (x1x * x1x + x1y * x1y) / (2.0 * r0 * r0);",
        "const double dph_common = k * sz - k - k * (x1x * x1x + x1y * x1y) / (2.0 * r0 * r0);"),
    "grad_drop_incident_depth": (
        "const double dph_common = k * sz - k + k * (x1x * x1x + x1y * x1y) / (2.0 * r0 * r0);",
        "const double dph_common = k * (x1x * x1x + x1y * x1y) / (2.0 * r0 * r0);"),
    "grad_cross_sign": (
        "const double dph = dph_common - k * (x1x * x2x + x1y * x2y) / (r0 * r0);",
        "const double dph = dph_common + k * (x1x * x2x + x1y * x2y) / (r0 * r0);"),
    "grad_unconjugated_phase": (
        "const double t_im = og[2 * i + 1] * c - og[2 * i] * s;",
        "const double t_im = og[2 * i + 1] * c + og[2 * i] * s;"),
    "grad_d1_wrong_part": (
        "gd1[n] = w * (d_re * (-ui) + d_im * ur);",
        "gd1[n] = w * (d_re * ur + d_im * ui);"),
    "grad_outer_unconjugated": (
        "og[2 * i + 1] = o_re * gu2[2 * i + 1] - o_im * gu2[2 * i];",
        "og[2 * i + 1] = o_re * gu2[2 * i + 1] + o_im * gu2[2 * i];"),
    "grad_drop_weight": (
        "gu1[2 * n] = w * s_re;\n            gu1[2 * n + 1] = w * s_im;",
        "gu1[2 * n] = s_re;\n            gu1[2 * n + 1] = s_im;"),
}


@pytest.mark.parametrize("name", sorted(GRAD_MUTANTS))
def test_planted_mistake_in_gradient_fails_a_pin(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "asfd_oracle.c")).read()
    old, new = GRAD_MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(src.replace(old, new, 1))
    lib = oracle.bind(oracle.compile_c(str(cpath), str(tmp_path / "libmutant.so")))
    errs = _grad_errors(lib)
    failures = [n for n, tol in GRAD_TOL.items() if not errs[n] < tol]
    assert failures, f"mutant {name} passed every gradient pin: {errs}"
