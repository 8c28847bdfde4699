"""Host-side arithmetic of `bench.py` that the JSON line reports: where the
roofline's DRAM traffic comes from (an ncu capture, only while the kernel's
sources and launch grid are the captured ones) and the fractions of the
on-chip resource peaks.  Nothing here needs a GPU."""
from __future__ import annotations

import math
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


KEY = ("spread_es_dense_kernel<7>", "smooth_random2048")


def test_captured_traffic_provenance(monkeypatch):
    rec = bench.NCU_TRAFFIC[KEY]
    # the record names a committed capture summary
    assert os.path.exists(os.path.join(ROOT, rec["capture"]))
    # unknown kernel or workload: no traffic
    assert bench.captured_traffic("other_kernel", KEY[1], rec["grid"])[0] is None
    assert bench.captured_traffic(KEY[0], "other_workload", rec["grid"])[0] is None
    # a different launch grid: no traffic, and the note says why
    val, note = bench.captured_traffic(KEY[0], KEY[1], rec["grid"] + 1)
    assert val is None and "grid" in note
    # sources that hash to the captured state: the captured bytes
    monkeypatch.setattr(bench, "sources_sha1", lambda paths: rec["sources_sha1"])
    val, note = bench.captured_traffic(KEY[0], KEY[1], rec["grid"])
    assert val == rec["bytes"] and rec["capture"] in note
    # changed sources: no traffic
    monkeypatch.setattr(bench, "sources_sha1", lambda paths: "0" * 40)
    val, note = bench.captured_traffic(KEY[0], KEY[1], rec["grid"])
    assert val is None and "changed" in note


def test_sources_hash_covers_the_spread_sources():
    h = bench.sources_sha1(bench.SPREAD_SOURCES)
    assert len(h) == 40 and int(h, 16) >= 0
    assert all(os.path.exists(os.path.join(ROOT, p)) for p in bench.SPREAD_SOURCES)


def test_resource_fractions_arithmetic():
    """Each fraction is the stage's algorithmic work over its time and the
    measured peak: 4 W^2 flops and 4 W exp2 evaluations per sample, W cells
    of 8 bytes per flushed window row (alpha_y n1y + W runs rows per source
    column), and (passes - 1) shared-memory stores and loads of each line."""
    g = dict(n1x=2048, n1y=2048, p1x=4e-6, p1y=4e-6, m2x=2048, m2y=2048, p2x=4e-6, p2y=4e-6,
             lam=633e-9, z0=0.1)
    info = {"nfx": 4096, "nfy": 4096, "run_rows": 36, "band_y0": 960, "band_y1": 3136}
    peaks = {"smem_load": {"value": 40000.0}, "smem_store": {"value": 34000.0},
             "l2_red_v2f32": {"value": 6000.0}, "ffma2": {"value": 80.0},
             "mufu_ex2": {"value": 10000.0}}
    stage_ms = [0.070, 0.029, 0.037]
    w = 7
    r = bench.resource_fractions(info, g, w, stage_ms, peaks)
    n = 2048 * 2048
    t_sp, t_r, t_c = 70e-6, 29e-6, 37e-6
    assert r["spread"]["ffma2"] == pytest.approx(4 * w * w * n / t_sp / 80e12)
    assert r["spread"]["mufu"] == pytest.approx(4 * w * n / t_sp / 10000e9)
    alpha_y = 4e-6 * 4e-6 * 4096 / (633e-9 * 0.1)
    runs = math.ceil(2048 / 36)
    flushed = 2048 * (alpha_y * 2048 + runs * w) * w * 8.0
    assert r["spread"]["l2_red"] == pytest.approx(flushed / t_sp / 6000e9)
    # 4096-point lines: three radix-16 passes, two exchanges through shared memory
    rows = 3136 - 960
    sm_r = 2 * 8.0 * 4096 * rows
    assert r["fft_rows"]["smem"] == pytest.approx((sm_r / 34000e9 + sm_r / 40000e9) / t_r)
    sm_c = 2 * 8.0 * 4096 * 2048
    assert r["fft_cols"]["smem"] == pytest.approx((sm_c / 34000e9 + sm_c / 40000e9) / t_c)
