"""Independent FP64 CPU oracle for the PP-WCNS-IS right-hand side.

TEST INFRASTRUCTURE: only the test-suite, ``__graft_entry__.smoke()``, the
benchmark's CPU-baseline legs and reference arm, and ``opcount_table.py``
(which writes the benchmark's stored operation counts) may import this
package.  It shares no code with the CUDA library.
"""
from .oracle import Oracle, OracleStats, build_oracle  # noqa: F401
