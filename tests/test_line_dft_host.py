"""The register DFTs (every pruning plan: butterflies, direct sums, Good-Thomas
and Cooley-Tukey splits) and the cooperative line DFT of every compiled line
shape, checked on the host against a direct FP64 DFT (tests/line_dft_host.cu,
compiled by nvcc as host code; no GPU)."""
import hashlib
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "line_dft_host.cu")
HDR = os.path.join(ROOT, "paper_2604_02624_gb300", "csrc", "dos_fft.cuh")
BUILD = os.path.join(ROOT, "tests", "_build")


def _binary():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    key = hashlib.sha1(open(SRC, "rb").read() + open(HDR, "rb").read()).hexdigest()[:16]
    exe = os.path.join(BUILD, f"line_dft_host_{key}")
    if not os.path.exists(exe):
        os.makedirs(BUILD, exist_ok=True)
        cmd = [nvcc, "-std=c++17", "--expt-relaxed-constexpr", "-O1", "-x", "cu", SRC, "-o", exe + ".tmp"]
        p = subprocess.run(cmd, capture_output=True, text=True)
        assert p.returncode == 0, p.stdout + p.stderr
        os.replace(exe + ".tmp", exe)
    return exe


def test_register_and_line_dfts_match_a_direct_fp64_dft():
    p = subprocess.run([_binary()], capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stdout + p.stderr
    assert p.stdout.strip().startswith("OK"), p.stdout
