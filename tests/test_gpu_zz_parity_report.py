"""Report of the FP64 parity cases that needed the conditioning fallback.

Collected after every other GPU parity module (test_gpu_*), it prints each
case whose error exceeded 1e-12 with its error, the oracle's 1-ulp spread
at the same input and the ratio of the two, and checks the recorded cases
against their bar once more: at most 4x the spread and below 1e-9.
"""
import pytest

from tests import parity_log

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def test_parity_fallback_report():
    for line in parity_log.summary_lines():
        print(line)
    for r in parity_log.RECORDS:
        for e, f in zip(r["err"], r["floor"]):
            assert e < 1e-9 and e <= max(r["tol"], 4.0 * f), r
