"""The package has no CPU path: with the compiled library missing, a call
through the public binding raises instead of computing anything (CPU, in a
fresh interpreter so that no library is loaded yet)."""
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROBE = r"""
from paper_2403_16862_gb300 import _binding as B
B.load.__defaults__ = ("/nonexistent/libinpc.so",)
try:
    B.inpc_sample_workspace_size(4096, 1000)
except ImportError as e:
    print("raised:", e)
else:
    print("computed without the library")
"""


def test_missing_library_raises():
    r = subprocess.run([sys.executable, "-c", PROBE], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr
    assert r.stdout.startswith("raised:") and "not built" in r.stdout, r.stdout
