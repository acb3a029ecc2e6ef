"""bench.py's modes that have no CPU arm answer with an `unavailable` line and
exit 0 without touching a GPU, as the reference arm's contract asks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def run_bench(*args):
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), *args], cwd=ROOT,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


@pytest.mark.parametrize("args", [
    ("--persistence-only", "--impl", "reference"),
    ("--persistence-only", "--workload", "serve"),
    ("--persistence-only", "--workload", "batch256"),
    ("--workload", "serve", "--impl", "reference"),
    ("--workload", "index512", "--impl", "reference"),
    ("--workload", "batch256", "--impl", "reference"),
])
def test_modes_without_a_cpu_arm_say_so(args):
    line = run_bench(*args)
    assert "unavailable" in line and line["unavailable"]
    assert line["impl"] == ("reference" if "reference" in args else "ours")
