"""Algorithmic operation counts of one RHS evaluation, per cell and
direction and per step of the method, from the oracle's op-counting build.

TEST INFRASTRUCTURE.  This script writes profiles/opcounts.json, the table
the benchmark's roofline lines read (the benchmark itself does not run the
oracle for it); tests/test_bench_roofline.py recomputes the table here and
requires the stored one to match.  Run from the repository root:

    python -m oracle.opcount_table

Three tables:
  shock_bubble_2d     the 2D shock / air-bubble workload on a 128 x 64 copy
                      (the benchmark grids are 1024 x 512 and 2048 x 1024;
                      the mix is per cell), one RHS at its CFL-0.5 dt;
  riemann_batch       16 seeded problems of the 4096-problem Riemann batch,
                      one RHS each at its CFL-0.5 dt, summed over their cells;
  bubble_collapse_3d  the 3D bubble collapse on a 24^3 copy (the workload is
                      384^3), one RHS at its CFL-0.5 dt.
Each table also holds the SSPRK3 stage combinations (Sec. 5.3), counted on
one step and given per stage (the sweeps fuse them into their last
direction).  The IS weights are counted in their one-division form (Sec. 4.3): the
oracle forms them with five ratio divisions and four normalising divisions
as printed; scaling every eta_k by the product of the five (beta + eps)
needs one division and 14 multiplications instead.
"""
import json
import os

import numpy as np

from oracle import Oracle
from paper_2102_05287_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
TABLE = os.path.join(ROOT, "profiles", "opcounts.json")
KEYS = ("add", "mul", "div", "sqrt", "minmax")


def _combine_row(o, W, dt, stages_units):
    """The SSPRK3 stage combinations (Sec. 5.3) of one counted step, per
    cell-stage and direction: the combine row of rk3_step over 3 x
    cells x directions."""
    o.opcount_reset()
    o.rk3_step(W, dt)
    c = o.opcount_rows()["ssprk3_combine"]
    return {k: c[k] / stages_units for k in KEYS}


def _one_division_form(per_step, is_calls):
    per_step["wcns_is"]["div"] -= 8 * is_calls
    per_step["wcns_is"]["mul"] += 14 * is_calls


def _table(per_step, is_calls, source):
    ops = {k: sum(c[k] for c in per_step.values()) for k in KEYS}
    ops["is_interpolations"] = is_calls
    ops["per_step"] = per_step
    ops["source"] = source
    return ops


def shock_bubble_2d(nx=128, ny=64):
    pr = P.shock_bubble_2d(nx, ny)
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, counting=True, **pr.eos)
    sm = o.max_wavespeed(pr.W)
    dt = 0.5 / (sm[0] * pr.n[0] / 2.0 + sm[1] * pr.n[1])
    o.opcount_reset()
    o.rhs(pr.W, dt)
    units = pr.ncells * pr.ndim  # cell-direction updates
    per_step = {r: {k: v / units for k, v in c.items()} for r, c in o.opcount_rows().items()}
    is_calls = 2 * (pr.ndim + 4) * o.stats.midpoints / units
    _one_division_form(per_step, is_calls)
    per_step["ssprk3_combine"] = _combine_row(o, pr.W, dt, 3 * units)
    return _table(per_step, is_calls, "shock_bubble_2d %dx%d, one RHS at CFL 0.5 (and the SSPRK3 stage "
                                      "combinations of one step, per stage)" % (nx, ny))


def bubble_collapse_3d(n=24):
    pr = P.bubble_collapse_3d(n)
    o = Oracle(pr.n, pr.lo, pr.hi, pr.bcs, counting=True, **pr.eos)
    sm = o.max_wavespeed(pr.W)
    dt = 0.5 / sum(sm[d] * pr.n[d] / (pr.hi[d] - pr.lo[d]) for d in range(3))
    o.opcount_reset()
    o.rhs(pr.W, dt)
    units = pr.ncells * pr.ndim
    per_step = {r: {k: v / units for k, v in c.items()} for r, c in o.opcount_rows().items()}
    is_calls = 2 * (pr.ndim + 4) * o.stats.midpoints / units
    _one_division_form(per_step, is_calls)
    per_step["ssprk3_combine"] = _combine_row(o, pr.W, dt, 3 * units)
    return _table(per_step, is_calls, "bubble_collapse_3d %d^3, one RHS at CFL 0.5 (and the SSPRK3 stage "
                                      "combinations of one step, per stage)" % n)


def riemann_batch(nsample=16):
    rb = P.riemann_batch()
    picks = np.random.default_rng(1).choice(len(rb.sizes), nsample, replace=False)
    rows, cells, mids = {}, 0, 0
    comb = dict.fromkeys(KEYS, 0.0)
    for k in picks:
        n = int(rb.sizes[k])
        W0 = np.ascontiguousarray(rb.W[:, int(rb.offsets[k]):int(rb.offsets[k + 1])])
        o = Oracle((n,), (0.0,), (1.0,), (("transmissive", "transmissive"),), counting=True, **rb.eos)
        dt = 0.5 / (o.max_wavespeed(W0)[0] * n)
        o.opcount_reset()
        o.rhs(W0, dt)
        for r, c in o.opcount_rows().items():
            acc = rows.setdefault(r, dict.fromkeys(KEYS, 0))
            for key, v in c.items():
                acc[key] += v
        cells += n
        mids += o.stats.midpoints
        for key, v in _combine_row(o, W0, dt, 3.0).items():
            comb[key] += v
    per_step = {r: {k: v / cells for k, v in c.items()} for r, c in rows.items()}
    is_calls = 2 * 5 * mids / cells
    _one_division_form(per_step, is_calls)
    per_step["ssprk3_combine"] = {k: v / cells for k, v in comb.items()}
    return _table(per_step, is_calls, "%d problems of the 4096-problem Riemann batch (%d cells), one RHS each "
                                      "at CFL 0.5" % (nsample, cells))


def compute_tables():
    return {"shock_bubble_2d": shock_bubble_2d(), "riemann_batch": riemann_batch(),
            "bubble_collapse_3d": bubble_collapse_3d()}


def main():
    with open(TABLE, "w") as f:
        json.dump(compute_tables(), f, indent=1, sort_keys=True)
        f.write("\n")
    print(TABLE)


if __name__ == "__main__":
    main()
