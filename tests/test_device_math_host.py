"""The device lens math compiled as host code (nvcc): the per-system-constant
EPL deflection equals the generic series, and its analytic vector-Jacobian
product equals forward-mode dual numbers and central differences."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_epl_vjp_host(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "epl_check"
    subprocess.run([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_2606_30620_b300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "epl_vjp_check.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    val, dual, fd, tail = float(out[1]), float(out[3]), float(out[5]), float(out[7])
    assert val < 1e-13 and dual < 1e-12 and fd < 1e-7, out
    # the early-exit bound of the forward render holds, and split sums are exact
    assert tail <= 1.0, out


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="nvcc not available")
def test_multiply_shift_division_is_exact(tmp_path):
    """The kernels split ray, pixel and cell indices with a multiply-high
    divider; its quotients equal integer division exactly."""
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    exe = tmp_path / "udiv_check"
    subprocess.run([nvcc, "-std=c++17", "-O2", "-I", os.path.join(ROOT, "paper_2606_30620_b300", "csrc"),
                    os.path.join(ROOT, "tests", "host", "udiv_check.cu"), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    assert int(out[1]) > 5_000_000 and int(out[3]) == 0, out
