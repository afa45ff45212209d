"""Host-side invariants of the team FFT's exchange layout and thread maps
(paper_2103_01767_gb300/csrc/team_fft.cuh) for all five FFT tiles: tests/fft_layout_check.cu,
compiled with nvcc for the host and run here (no GPU).  It checks that exchange 1's words
are distinct and read back as the decomposition needs, that exchange 2 stays inside warps
and covers every value once, that every warp access of the three passes is free of
shared-memory bank conflicts (16 distinct bank pairs per half-warp), and that the pass-3
frequency map is a bijection that freq_place inverts."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.skipif(shutil.which("nvcc") is None, reason="nvcc not on PATH")
def test_exchange_layout_and_maps(tmp_path):
    exe = tmp_path / "fft_layout_check"
    src = os.path.join(ROOT, "tests", "fft_layout_check.cu")
    inc = os.path.join(ROOT, "paper_2103_01767_gb300", "csrc")
    subprocess.run(["nvcc", "-std=c++17", "-O1", "-I", inc, "-o", str(exe), src], check=True, capture_output=True,
                   timeout=300)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    lines = r.stdout.strip().splitlines()
    assert len(lines) == 5, r.stdout + r.stderr
    for line in lines:
        assert line.endswith(": 0 failed checks"), line
    assert r.returncode == 0
