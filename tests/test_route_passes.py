"""Pass routing (which buffer each scatter pass reads and writes, and whether
a final copy is needed) checked exhaustively on the host: every pass count up
to the maximum, every pattern of trivial passes, in place and out of place.
The routing function is compiled for the host by nvcc; nothing runs on a GPU."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def test_every_pattern_of_skipped_passes_routes_correctly(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    exe = str(tmp_path / "route_check")
    subprocess.run([nvcc, "-std=c++17", "-O1", "-o", exe, os.path.join(HERE, "route_check.cu")], check=True,
                   capture_output=True)
    p = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stdout[-2000:]
    cases = 2 * sum(1 << j for j in range(17))  # passes 0..16, every mask, in place or not
    assert f"cases {cases} bad 0" in p.stdout
