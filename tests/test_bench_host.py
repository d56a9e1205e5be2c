"""CPU tests of bench.py's host logic: the clock record that decides whether a
timed run is kept (throttle reasons, median SM clock under load) and the
algorithmic byte and flop counts the roofline fractions divide by."""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


def test_clock_summary_reads_reasons_per_device(tmp_path):
    """nvidia-smi rows (index, clocks.sm, clocks.max.sm, power, active mask,
    hw_slowdown, hw_thermal_slowdown, sw_thermal_slowdown, sw_power_cap): the
    summary takes the median SM clock and the reasons seen Active, for the
    bench's own device only; "Not Active" is not a reason, and rows cut short
    or unreadable are skipped."""
    rows = [
        "0, 2070, 2070, 900.1, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "1, 1200, 2070, 300.0, 0x0000000000000008, Active, Not Active, Not Active, Not Active",
        "0, 2055, 2070, 1350.0, 0x0000000000000004, Not Active, Not Active, Not Active, Active",
        "0, 2070, 2070, 1200.5, 0x0000000000000000, Not Active, Not Active, Not Active, Not Active",
        "0, [N/A], 2070, 0, 0x0, Not Active",
        "",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    c = bench.ClockSampler(str(path))
    s0 = c.summary(0)
    assert s0["sm_mhz"] == 2070.0 and s0["sm_max_mhz"] == 2070.0
    assert s0["reasons"] == ["sw_power_cap"]
    assert s0["samples"] == 4
    s1 = c.summary(1)
    assert s1["sm_mhz"] == 1200.0 and s1["reasons"] == ["hw_slowdown"]
    assert bench.ClockSampler(str(tmp_path / "absent.csv")).summary(0)["sm_mhz"] is None


def _toy_plan(rows=((6, 9, 13, 4096, 500_000), (5, 13, 21, 512, 120_000), (4, 21, 37, 64, 2_000))):
    info = {"n_unknowns": 30_000, "n_triangles": 20_000, "moment_entries_rwg": 3_000_000,
            "moment_entries_tri": 1_800_000, "near_nnz_A": 4.0e7, "near_nnz_V": 1.7e7}
    levels = [{"level": l, "sp": sp, "nfft": n, "n_boxes": b, "n_far_pairs": fp} for l, sp, n, b, fp in rows]
    return info, levels


def test_grid_bytes_count_setup_products_once_per_batch():
    """Grids, spectra and vectors grow with the right-hand sides of a batch;
    the moments (a setup product) are counted once per batch, so doubling the
    batch doubles every class's bytes less the moment bytes."""
    info, levels = _toy_plan()
    mom = (3 * info["moment_entries_rwg"] + info["moment_entries_tri"]) * 4
    for vb in (8, 16):
        mom_vb = (3 * info["moment_entries_rwg"] + info["moment_entries_tri"]) * (vb // 2)
        g32, g64 = bench.grid_bytes(info, levels, 32, vb), bench.grid_bytes(info, levels, 64, vb)
        for name in ("anterpolation", "interpolation"):
            assert np.isclose(2 * g32[name] - g64[name], mom_vb), name
        for name in ("forward_fft", "inverse_fft", "upward", "downward"):
            assert np.isclose(2 * g32[name], g64[name]), name
    assert mom == (3 * 3_000_000 + 1_800_000) * 4
    # the transfers run between grid levels only: one level, no transfer bytes
    one = bench.grid_bytes(info, levels[:1], 8, 8)
    assert one["upward"] == 0 and one["downward"] == 0


def test_algorithmic_counts():
    """Translation flops: 8 per complex multiply-add, pairs x n^3 per channel,
    4 channels per right-hand side, the top grid level apart from the
    interaction-list levels; near field: 8 flops per stored entry per
    right-hand side and 16 bytes per entry once per batch."""
    info, levels = _toy_plan()
    a = bench.algorithmic({}, info, levels, 64)
    top = 8.0 * 2_000 * 37 ** 3 * 4 * 64
    il = 8.0 * (500_000 * 13 ** 3 + 120_000 * 21 ** 3) * 4 * 64
    assert np.isclose(a["translation_mac_top"][1], top) and np.isclose(a["translation_mac_top_tc"][1], top)
    assert np.isclose(a["translation_mac"][1], il) and np.isclose(a["translation_mac_tc"][1], il)
    assert np.isclose(a["near_A"][1], 8.0 * 4.0e7 * 64) and np.isclose(a["near_V"][1], 8.0 * 1.7e7 * 64)
    a1 = bench.algorithmic({}, info, levels, 1)
    assert a1["near_A_bytes"] == a["near_A_bytes"] == 16.0 * 4.0e7


def test_oracle_rate_aggregation():
    """The reference arm's rate: matvec fractions (seconds taken / estimated
    seconds of one matvec) completed by all workers, over the wall time."""
    res = [{"est": [10.0, 10.0], "took": [1.0, 2.0]}, {"est": [4.0], "took": [1.0]}]
    assert np.isclose(bench._oracle_rates(res, 2.0), (0.1 + 0.2 + 0.25) / 2.0)
