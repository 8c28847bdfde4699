"""The 1D oracle against its pins (tests/oracle_line_pins.py), and planted
mistakes in its C source that must fail at least one pin."""
from __future__ import annotations

import os

import pytest

import oracle
from oracle import line as oline
from tests import oracle_line_pins as pins


def _fn(lib=None):
    def f(g, x1, d1, w, u1, form):
        return oline.line(g, x1, d1, w, u1, form, lib=lib)
    return f


@pytest.mark.parametrize("name", sorted(pins.LINE_PINS))
def test_line_pin(name):
    fn, tol = pins.LINE_PINS[name]
    err = fn(_fn())
    assert err < tol, f"{name}: {err:.3e} >= {tol:.1e}"


MUTANTS = {
    "cross_sign": ("- k * x * x2 / r0;", "+ k * x * x2 / r0;"),
    "chirp_z0": ("ph = ph_inc + k * (-h + x * x / (2.0 * r0))", "ph = ph_inc + k * (-h + x * x / (2.0 * g->z0))"),
    "dest_chirp_z0": ("if (form == 5) ph += k * x2 * x2 / (2.0 * r0);",
                      "if (form == 5) ph += k * x2 * x2 / (2.0 * g->z0);"),
    "prefactor_no_sqrt": ("f = 1.0 / sqrt(g->lambda * g->z0);", "f = 1.0 / (g->lambda * g->z0);"),
    "huygens_exponent": ("amp /= r * sqrt(r);", "amp /= r * r;"),
    "drop_weight": ("double ph, amp = w[j];", "double ph, amp = 1.0;"),
    "tilt_sign": ("const double ph_inc = k * (g->s * x + sz * h);",
                  "const double ph_inc = k * (-g->s * x + sz * h);"),
    "quarter_turn_sign": ("ph0 = k * g->z0 - 0.25 * LINE_PI;", "ph0 = k * g->z0 + 0.25 * LINE_PI;"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_line_pin(name, tmp_path):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "asfd_oracle_line.c")).read()
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation anchor for {name} not unique"
    cpath = tmp_path / "mutant.c"
    cpath.write_text(src.replace(old, new, 1))
    lib = oline.bind(oracle.compile_c(str(cpath), str(tmp_path / "libmutant.so")))
    failures = [p for p, (fn, tol) in pins.LINE_PINS.items() if not fn(_fn(lib)) < tol]
    assert failures, f"mutant {name} passed every pin"
