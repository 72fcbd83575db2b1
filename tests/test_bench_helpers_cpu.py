"""The benchmark's own input preparation and record arithmetic (CPU only):
the periodic ghost fill it gives the oracle equals the oracle's fill, the
1024^3 level's groups map onto the periodic 256^3 field they repeat, and the
roofline records divide what they say they divide."""
from __future__ import annotations

import importlib.util
import os

import numpy as np
import pytest

import oracle
from paper_1007_3818_gb300 import workloads as wl

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


@pytest.mark.parametrize("n", [32, 64])
def test_periodic_tiles_equal_the_oracle_fill(bench, n):
    gx = n // 16
    groups = wl.level_to_groups(wl.fourier_level(n=n, seed=n, gamma=5 / 3))
    want = oracle.fill_ghosts_uniform(groups, gx, gx, gx, 0)
    got = bench.periodic_tiles(groups, gx)
    assert np.array_equal(got, want)
    # the reused output buffer gives the same result
    assert np.array_equal(bench.periodic_tiles(groups, gx, out=np.empty_like(want)), want)


def test_tiled_level_groups_map_onto_the_periodic_field(bench):
    """Group (bx, by, bz) of the 64^3-group level is group (bx mod 16, by mod
    16, bz mod 16) of the 16^3-group field; every field group appears 64 times."""
    src = bench.tiled_sources(64, 16)
    g = np.arange(64 ** 3)
    bx, by, bz = g % 64, (g // 64) % 64, g // 4096
    assert np.array_equal(src, ((bz % 16) * 16 + by % 16) * 16 + bx % 16)
    assert np.array_equal(np.bincount(src), np.full(4096, 64))
    # neighbours across a repeat boundary are the field's periodic neighbours
    assert src[15] == 15 and src[16] == 0


def test_roofline_records(bench):
    peaks = {"f32": 80.0, "f64": 1.25, "f32_at_median_clock": 64.0, "f64_at_median_clock": 1.0,
             "basis_f32": "b32", "basis_f64": "b64"}
    rl = bench.rooflines(1000.0, 4096 * 100, 2.0, 4, peaks, 6000.0, None, "f32", "k")
    ach = 1000.0 * 4096 * 100 / 2e-3 / 1e12
    assert rl["alu"]["achieved"] == pytest.approx(ach)
    assert rl["alu"]["frac"] == pytest.approx(ach / 80.0)
    assert rl["alu"]["frac_of_lane_op_peak"] == pytest.approx(2 * ach / 80.0)
    assert rl["alu"]["frac_at_median_clock"] == pytest.approx(ach / 64.0)
    nbytes = 100 * ((20480 * 2 + 7680) * 4 + 68)
    assert rl["hbm"]["algorithmic_bytes"] == nbytes
    assert rl["hbm"]["frac"] == pytest.approx(nbytes / 2e-3 / 1e9 / 6000.0)
    f64 = bench.rooflines(1000.0, 4096, 1.0, 8, peaks, 6000.0, None, "f64", "k")
    assert f64["alu"]["peak"] == 1.25
    assert bench.rooflines(None, 4096, 1.0, 4, peaks, 6000.0, None, "f32", "k").get("alu") is None


def test_traffic_figure_only_for_the_profiled_sources(bench, monkeypatch):
    t = bench.NCU_TRAFFIC
    assert bench.measured_traffic("f32", t["groups"]) in (None, t["bytes"])
    if bench.measured_traffic("f32", t["groups"]) is not None:
        assert bench.measured_traffic("f32", 64 * t["groups"]) == 64 * t["bytes"]
    assert bench.measured_traffic("mixed", t["groups"]) is None
    monkeypatch.setattr(bench, "kernel_sources_sha256", lambda: "0" * 64)
    assert bench.measured_traffic("f32", t["groups"]) is None
