"""Build ``libisofft.so`` (the C-ABI library of include/isofft.h) in-tree.

Every CUDA translation unit is compiled for sm_103a only, in parallel, then
linked into ``paper_1106_0557_gb300/libisofft.so``.  Objects go to
``_build/`` at the repository root.  nvcc cross-compiles, so this runs on a
host without a GPU; on an aarch64 GPU host the same command builds natively.
"""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libisofft.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
         "-I", INCLUDE, "-I", CSRC]


def _spectrum_code():
    """32-bit digest of the sources that define the cached Green's spectrum
    (its build and layout); spectrum files written by other code are
    rejected (see ISOFFT_SPECTRUM_DIR in include/isofft.h)."""
    import hashlib
    h = hashlib.sha256()
    for fn in ("greens.cu", "launch.h", "fft_engine.cuh", "passes.cuh"):
        with open(os.path.join(CSRC, fn), "rb") as f:
            h.update(f.read())
    return "0x%08x" % (int(h.hexdigest()[:8], 16) | 1)


def _units():
    units = [("api", "api.cu", ["-DISOFFT_SPECTRUM_CODE=%s" % _spectrum_code()]), ("greens", "greens.cu", []),
             ("noalloc", "noalloc.cu", []), ("batch", "batch.cu", [])]
    for real, tag in (("float", "f32"), ("double", "f64"), ("isofft::df64", "df64")):
        for group, gname in ((1, "x"), (2, "y"), (3, "z")):
            units.append(("passes_%s_%s" % (gname, tag), "passes_inst.cu",
                          ["-DISOFFT_REAL=%s" % real, "-DISOFFT_GROUP=%d" % group]))
    return units


def _sources():
    return (glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cuh"))
            + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
            + [os.path.abspath(__file__)])


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def _nvcc():
    nv = shutil.which("nvcc")
    if nv:
        return nv
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libisofft")


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)

    def compile_one(u):
        name, src, defs = u
        obj = os.path.join(BUILD, name + ".o")
        cmd = [nvcc] + ARCH + FLAGS + defs + ["-c", os.path.join(CSRC, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (name, " ".join(cmd), r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    units = _units()
    workers = max(1, min(len(units), os.cpu_count() or 1))
    with cf.ThreadPoolExecutor(workers) as ex:
        objs = list(ex.map(compile_one, units))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s\n%s" % (" ".join(cmd), r.stderr))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
