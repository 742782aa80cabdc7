import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300) and the built CUDA library")
    config.addinivalue_line("markers", "slow: long-running CPU test")


def load_golden(name):
    rows = []
    with open(os.path.join(ROOT, "tests", "golden", name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([float(x) for x in line.split()])
    return rows


def build_abi_consumer(libpath, outdir):
    """Compile tests/abi_consumer.c as strict C99 against include/wcns.h and
    the built libwcns.so; returns the executable's path."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.dirname(os.path.abspath(libpath))
    exe = os.path.join(str(outdir), "abi_consumer")
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-O2",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", "abi_consumer.c"),
           "-L", libdir, "-lwcns", "-Wl,-rpath," + libdir, "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def pytest_terminal_summary(terminalreporter, exitstatus, config):
    """Report the FP64 parity cases that needed the conditioning fallback."""
    try:
        from tests import parity_log
    except Exception:
        return
    if "tests.test_gpu_parity" in sys.modules or "test_gpu_parity" in sys.modules:
        terminalreporter.write_sep("-", "FP64 parity fallback report")
        for line in parity_log.summary_lines():
            terminalreporter.write_line(line)
