"""Host-side roofline arithmetic of bench.py (CPU).

The FP64 line counts the oracle's per-step operation mix (IS weights in
their one-division form) at the measured FP64 peak; the mixed line puts the
steps the mixed sweeps compute in FP64 (node EOS, node fluxes, update) at
the FP64 peak and all others at the FP32 peak.  These tests pin that
bookkeeping: the per-step counts add up to the totals the FP64 roofline
uses, the one-division adjustment touches only the WCNS-IS step, the mixed
fraction equals the two pipe times over the launch time, and the stored
tables (profiles/opcounts.json) are what the oracle gives.
"""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import bench  # noqa: E402


@pytest.fixture(scope="module")
def ops():
    return bench.algorithmic_ops(128, 64)


def test_per_step_counts_add_up_to_the_totals(ops):
    for k in ("add", "mul", "div", "sqrt", "minmax"):
        total = sum(c[k] for c in ops["per_step"].values())
        assert total == pytest.approx(ops[k], rel=1e-12), k


def test_one_division_form_only_changes_wcns_is(ops):
    n_is = ops["is_interpolations"]
    # two interpolations per field (six in 2D) and midpoint; the counting
    # grid is 128 x 64, whose lines have n + 1 midpoints for n cells
    nx, ny = 128, 64
    midpoints = ny * (nx + 1) + nx * (ny + 1)
    assert n_is == pytest.approx(2 * 6 * midpoints / (2 * nx * ny), rel=1e-12)
    # one division per interpolation left in the WCNS-IS step
    assert ops["per_step"]["wcns_is"]["div"] == pytest.approx(n_is, rel=1e-12)
    assert ops["per_step"]["projection"]["div"] > 0


def test_mixed_roofline_is_two_pipe_time_over_launch_time(ops):
    peaks = {"fp64_fma_tflops": 1.25, "fp32_fma_tflops": 75.0}
    ncell, ms = 524288, 0.1
    r = bench.mixed_roofline(ops, peaks, ms, ncell, fallbacks=0)
    f64 = sum(sum(c.values()) for s, c in ops["per_step"].items() if s in bench.MIXED_FP64_STEPS)
    f32 = sum(sum(c.values()) for s, c in ops["per_step"].items() if s not in bench.MIXED_FP64_STEPS)
    assert r["fp64_flops_per_cell_dir"] == pytest.approx(f64)
    assert r["fp32_flops_per_cell_dir"] == pytest.approx(f32)
    t64, t32 = f64 * ncell / 1.25e12, f32 * ncell / 75e12
    assert r["frac"] == pytest.approx((t64 + t32) / (ms * 1e-3))
    assert r["frac_overlapped"] == pytest.approx(max(t64, t32) / (ms * 1e-3))
    # achieved / peak is the same fraction, in FP64-equivalent flop/s
    assert r["achieved"] / r["peak"] == pytest.approx(r["frac"])
    assert set(bench.MIXED_FP64_STEPS) <= set(ops["per_step"])


def test_stored_opcount_tables_match_the_oracle():
    """profiles/opcounts.json, which the benchmark reads, is what the
    oracle's op-counting build gives now (oracle/opcount_table.py)."""
    import json

    from oracle.opcount_table import TABLE, compute_tables
    with open(TABLE) as f:
        stored = json.load(f)
    fresh = json.loads(json.dumps(compute_tables()))
    assert stored == fresh
