"""The bounds-checked build of the library (every index the kernels compute into shared memory, x and y is
tested against its buffer; a violation is recorded as EHYB_ERR_BOUNDS and the access skipped) runs the parity
cases of every path without a report.  It stands in for a memory checker, which this pool does not offer."""
import importlib.util
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_checked_build_runs_every_path_without_a_bounds_report():
    spec = importlib.util.spec_from_file_location("ehyb_build", os.path.join(ROOT, "paper_2204_06666_gb300", "build.py"))
    builder = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(builder)
    lib = builder.build(checked=True)
    env = dict(os.environ, EHYB_LIBRARY=lib)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "tests", "checked_cases.py")], env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0 and "CHECKED OK" in r.stdout, r.stdout[-3000:] + r.stderr[-3000:]
