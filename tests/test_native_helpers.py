"""Host-side checks of the library's small native helpers (no GPU)."""
import os
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_fastdiv_matches_hardware_division():
    src = os.path.join(ROOT, "tests", "native", "fastdiv_check.cpp")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "fastdiv_check")
        subprocess.check_call(["g++", "-O2", "-std=c++17", src, "-o", exe])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr


def test_point_mean_rounding_is_exact():
    """The geometry kernel's narrow coordinate path, fl(o) + fl(k / n) with
    one fixed exception: the correctly rounded mean for every cell
    coordinate o below 2^21 and every corner count n and k."""
    src = os.path.join(ROOT, "tests", "native", "mean_rounding_check.c")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "mean_rounding_check")
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", src, "-o", exe, "-lm"])
        out = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0 and out.stdout.strip() == "ok", out.stdout + out.stderr
