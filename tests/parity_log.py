"""Record of the FP64 parity cases that needed the conditioning fallback.

assert_parity (tests/test_gpu_parity.py) asserts 1e-12 relative per field;
where a field exceeds it, the bar becomes 4x the oracle's own spread under
1-ulp input perturbations (the limiter theta solves and the IS weights next
to discontinuities amplify round-off).  Every such case is recorded here,
so that the session can report how often the fallback was needed and by
how much (tests/test_gpu_zz_parity_report.py, and the terminal summary
written by tests/conftest.py).
"""
RECORDS = []


def record(case, err, floor, tol):
    """One fallback: per-field errors, the oracle's 1-ulp spread, the bar."""
    RECORDS.append({"case": case, "err": [float(x) for x in err], "floor": [float(x) for x in floor],
                    "tol": float(tol)})


def summary_lines():
    if not RECORDS:
        return ["FP64 parity: every case within 1e-12 (no conditioning fallback needed)"]
    lines = ["FP64 parity cases above 1e-12 (bar: 4x the oracle's 1-ulp spread, and < 1e-9):"]
    worst = max(RECORDS, key=lambda r: max(r["err"]))
    for r in RECORDS:
        e = max(r["err"])
        k = r["err"].index(e)
        lines.append("  %-70s max err %.2e (field %d)  1-ulp spread %.2e  err/1e-12 %.0f  err/spread %.2f" %
                     (r["case"][:70], e, k, r["floor"][k], e / r["tol"], e / max(r["floor"][k], 1e-300)))
    lines.append("  %d case(s); worst %.2e = %.0f x 1e-12 (%s)" %
                 (len(RECORDS), max(worst["err"]), max(worst["err"]) / worst["tol"], worst["case"]))
    return lines
