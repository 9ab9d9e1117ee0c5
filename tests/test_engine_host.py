"""The FFT engine's stage code on the CPU, against a direct DFT.

fft_engine.cuh is host-callable; engine_host_check.cu drives every line
shape the passes instantiate through the same stage, butterfly and root
code, in FP32, FP64 and float pairs, and
compares with a long-double DFT.
No GPU: nvcc compiles host code only here.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1106_0557_gb300", "csrc")
BUILD = os.path.join(ROOT, "_build")

# error bounds relative to max |X|: a few units of roundoff times log2 L
TOL = {"f32": 5e-7, "f64": 2e-15, "df64": 3e-14}


def _nvcc():
    nv = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nv):
        pytest.skip("nvcc not available")
    return nv


@pytest.fixture(scope="module")
def engine_errors():
    os.makedirs(BUILD, exist_ok=True)
    exe = os.path.join(BUILD, "engine_host_check")
    src = os.path.join(HERE, "engine_host_check.cu")
    deps = [src] + [os.path.join(CSRC, f) for f in ("fft_engine.cuh", "df64.cuh")]
    if not os.path.exists(exe) or os.path.getmtime(exe) < max(os.path.getmtime(d) for d in deps):
        subprocess.run([_nvcc(), "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, "-o", exe, src],
                       check=True)
    out = subprocess.run([exe], check=True, capture_output=True, text=True).stdout
    errs = {}
    for line in out.strip().splitlines():
        name, val = line.split()
        errs[name] = float(val)
    return errs


def test_engine_covers_every_shape_and_dtype(engine_errors):
    for tag in TOL:
        names = [n for n in engine_errors if "_%s_" % tag in n]
        assert len(names) >= 44, (tag, len(names))


@pytest.mark.parametrize("tag", sorted(TOL))
def test_engine_matches_direct_dft(engine_errors, tag):
    bad = {n: e for n, e in engine_errors.items() if "_%s_" % tag in n and not e <= TOL[tag]}
    assert not bad, bad


def test_float_pairs_beat_float_by_five_orders(engine_errors):
    for name, e in engine_errors.items():
        if "_df64_" in name and name.replace("_df64_", "_f32_") in engine_errors:
            e32 = engine_errors[name.replace("_df64_", "_f32_")]
            assert e * 1e5 < e32 * 10, (name, e, e32)
