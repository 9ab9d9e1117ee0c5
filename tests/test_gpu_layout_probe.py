"""The read pattern behind the z-blocked workspace (2304-point z lines).

stride_read_probe.cu reads a 12 GB array shaped like the 1152^3 workspace
in 32-byte chunks, once along z (the z pass's line groups) and once along y
(the y passes' columns), with the planes plain (zb = 1) or in blocks of 4
and 16.  Blocks of 16 planes put the z reads of a line group 9 KB apart
within a block instead of a whole 21 MB plane apart; the test checks that
this reads at least 1.5x faster along z, and that the y pattern keeps at
least half its plain rate.  The figures are printed for the record.
"""
import os
import shutil
import subprocess

import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(os.path.dirname(HERE), "_build")


def test_z_blocks_speed_up_the_z_read_pattern():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "stride_read_probe")
    subprocess.run([nv, "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-o", exe,
                    os.path.join(HERE, "stride_read_probe.cu")], check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True, timeout=120).stdout
    gbs = {}
    for line in out.split("\n"):
        if line.strip():
            zb, pat, v = line.split()
            gbs[(int(zb), pat)] = float(v)
    print("strided 32-byte reads, GB/s:", gbs)
    assert gbs[(16, "z")] >= 1.5 * gbs[(1, "z")]
    assert gbs[(16, "y")] >= 0.5 * gbs[(1, "y")]
