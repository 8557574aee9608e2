"""The bench's ALU roofline arithmetic (bench.roofline_of), on the CPU: the peak
of a batch is the rate at which its cells would run with each cell width at its
own measured peak (int32 cells at the two-pipe add/max rate, int16x2 cells at
twice the packed add-max lane rate), so a single-width batch reports that
width's peak, and a mix reports the cell-weighted harmonic mean of the two."""
import math

import pytest

import bench

PROBE = {"int_ops": 40e12, "viaddmax_s16x2_lanes": 40e12}  # packed peak 80 Tops/s


def test_single_width_peaks():
    cells, ms = 1e10, 10.0
    achieved = cells * 9 / (ms * 1e-3) / 1e12  # 9 Tops/s
    r = bench.roofline_of("protein-sw-100k", cells, 0, ms, PROBE, None)
    assert r["achieved"] == pytest.approx(achieved)
    assert r["peak"] == pytest.approx(40.0)
    assert r["frac"] == pytest.approx(achieved / 40.0)
    r = bench.roofline_of("protein-sw-100k", cells, cells, ms, PROBE, None)
    assert r["peak"] == pytest.approx(80.0)
    assert r["frac"] == pytest.approx(achieved / 80.0)
    assert r["cells"] == {"i32": 0, "i16x2": cells}


@pytest.mark.parametrize("f", [0.25, 0.5, 0.953])
def test_mixed_peak_is_the_cell_weighted_harmonic_mean(f):
    cells = 3e10
    r = bench.roofline_of("protein-sw-100k", cells, f * cells, 19.0, PROBE, None)
    want = 1.0 / ((1 - f) / 40.0 + f / 80.0)
    assert r["peak"] == pytest.approx(want)
    assert 40.0 < r["peak"] < 80.0


def test_recorded_protein_run():
    """The protein step of the last full bench run: 3.03e10 cells, 99.2% of them
    int16x2, forward 19.09 ms, probe rates 39.80 / 39.64 T: fraction 0.181."""
    probe = {"int_ops": 39796142868854.625, "viaddmax_s16x2_lanes": 39635323587844.38}
    r = bench.roofline_of("protein-sw-100k", 241278013 + 30038499365, 30038499365,
                          19.092479705810547, probe, 0.6097)
    assert r["achieved"] == pytest.approx(14.2736, rel=1e-4)
    assert r["peak"] == pytest.approx(78.649, rel=1e-4)
    assert r["frac"] == pytest.approx(0.18148, rel=1e-3)
    # DRAM bytes per step from the captured bytes per cell; algorithmic 0.5 B/cell
    assert r["traffic"] == pytest.approx(0.6097 * 30279777378)
    assert r["algorithmic_bytes"] == pytest.approx(0.5 * 30279777378)
    assert r["kernel"].startswith("k_full + k_pack")


def test_without_probe_or_capture():
    r = bench.roofline_of("long-reads-10k", 1e9, 0, 5.0, None, None)
    assert r["peak"] is None and r["frac"] is None and r["traffic"] is None
    assert r["kernel"].startswith("k_xdrop")
    assert math.isclose(r["forward_gcups"], 200.0)
