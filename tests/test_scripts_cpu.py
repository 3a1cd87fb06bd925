"""The package's command-line modules start and parse their arguments
without a GPU (their timed work needs one)."""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("mod", ["paper_2509_19974_gb300.workloads",
                                 "paper_2509_19974_gb300.accuracy_sweep"])
def test_module_help(mod):
    r = subprocess.run([sys.executable, "-m", mod, "--help"], capture_output=True, text=True,
                       timeout=120, cwd=ROOT)
    assert r.returncode == 0, r.stderr
    assert "usage" in r.stdout
