"""FP64 CPU oracle for the isolated-system Poisson solve (PSPFFT, Sec. 2).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the benchmark's
CPU-baseline leg may import this package.  It shares no code with the CUDA
library; the two meet only through the seeded source generators, which hold
none of the method's arithmetic.

Everything here is FP64 on the host:

* ``green``/``green_table``  -- Eq. 6 and the doubled-mesh table of Eq. 9,
* ``fft1d``/``fft3d``        -- the oracle's own recursive mixed-radix FFT,
* ``solve``                  -- route 2: pad, forward DFT, multiply by the
  transform of the Eq. 9 table (Eq. 5), inverse DFT, crop (Sec. 2.2.2),
* ``direct_sum``/``direct_points`` -- route 1: the discrete convolution
  summed cell by cell, the definition the mesh-doubling method reproduces
  exactly up to rounding (Sec. 2.1),
* ``analytic`` -- closed-form potentials of the test problems (Sec. 4).
"""
import ctypes
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        d = ctypes.c_double
        i64 = ctypes.c_int64
        p = ctypes.c_void_p
        L.oracle_green.restype = d
        L.oracle_green.argtypes = [ctypes.c_long, ctypes.c_long, ctypes.c_long, p]
        L.oracle_green_table.restype = None
        L.oracle_green_table.argtypes = [p, p, p]
        L.oracle_green_block.restype = None
        L.oracle_green_block.argtypes = [p, p, p, p]
        L.oracle_fft1d.restype = ctypes.c_int
        L.oracle_fft1d.argtypes = [p, i64, ctypes.c_int]
        L.oracle_fft3d.restype = ctypes.c_int
        L.oracle_fft3d.argtypes = [p, p, ctypes.c_int]
        L.oracle_green_spectrum.restype = ctypes.c_int
        L.oracle_green_spectrum.argtypes = [p, p, p]
        L.oracle_solve_with_spectrum.restype = ctypes.c_int
        L.oracle_solve_with_spectrum.argtypes = [p, p, p, p, p]
        L.oracle_solve.restype = ctypes.c_int
        L.oracle_solve.argtypes = [p, p, p, p, p]
        L.oracle_direct_point.restype = d
        L.oracle_direct_point.argtypes = [p, p, p, i64, i64, i64]
        L.oracle_direct_sum.restype = None
        L.oracle_direct_sum.argtypes = [p, p, p, p]
        L.oracle_direct_points.restype = None
        L.oracle_direct_points.argtypes = [p, p, p, p, i64, p]
        L.oracle_num_threads.restype = ctypes.c_int
        L.oracle_num_threads.argtypes = []
        _lib = L
    return _lib


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _i64(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.int64))


def _f64(v):
    return np.ascontiguousarray(np.asarray(v, dtype=np.float64))


def num_threads() -> int:
    return int(lib().oracle_num_threads())


def doubled_mesh(N):
    """The paper's doubled mesh, M = 2N per axis (Sec. 2.1)."""
    return tuple(2 * int(n) for n in N)


def green(d, h):
    """Eq. 6 at integer offset d = (dx, dy, dz); the origin takes the value
    Eq. 9 assigns to it."""
    hh = _f64(h)
    return float(lib().oracle_green(int(d[0]), int(d[1]), int(d[2]), _ptr(hh)))


def green_table(M, h):
    """Eq. 9 on the doubled mesh M: real array [Mz][My][Mx]."""
    MM, hh = _i64(M), _f64(h)
    out = np.empty((MM[2], MM[1], MM[0]), dtype=np.float64)
    lib().oracle_green_table(_ptr(MM), _ptr(hh), _ptr(out))
    return out


def green_block(lo, n, h):
    """Eq. 6 (Eq. 9 at the origin) at the offsets lo + [0, n) per axis: real
    array [n_z][n_y][n_x].  The corner-impulse response of a box, read in
    slabs at sizes where the doubled table would not fit in memory."""
    L0, NN, hh = _i64(lo), _i64(n), _f64(h)
    out = np.empty((NN[2], NN[1], NN[0]), dtype=np.float64)
    lib().oracle_green_block(_ptr(L0), _ptr(NN), _ptr(hh), _ptr(out))
    return out


def fft1d(x, inverse=False):
    """The oracle's recursive FFT of a 1-D complex array.  Forward uses
    e^{-2 pi i jk/n}; the inverse is unnormalised."""
    a = np.ascontiguousarray(np.asarray(x, dtype=np.complex128)).copy()
    rc = lib().oracle_fft1d(_ptr(a), a.size, 1 if inverse else -1)
    if rc:
        raise RuntimeError("oracle_fft1d failed: %d" % rc)
    return a


def fft3d(g, inverse=False):
    """3-D transform of a complex [Mz][My][Mx] array (x, y, z order forward,
    z, y, x inverse; the inverse is unnormalised)."""
    a = np.ascontiguousarray(np.asarray(g, dtype=np.complex128)).copy()
    M = _i64([a.shape[2], a.shape[1], a.shape[0]])
    rc = lib().oracle_fft3d(_ptr(a), _ptr(M), 1 if inverse else -1)
    if rc:
        raise RuntimeError("oracle_fft3d failed: %d" % rc)
    return a


def green_spectrum(M, h):
    """Transform of the Eq. 9 table divided by Mx My Mz: complex [Mz][My][Mx]."""
    MM, hh = _i64(M), _f64(h)
    out = np.empty((MM[2], MM[1], MM[0]), dtype=np.complex128)
    rc = lib().oracle_green_spectrum(_ptr(MM), _ptr(hh), _ptr(out))
    if rc:
        raise RuntimeError("oracle_green_spectrum failed: %d" % rc)
    return out


def solve_with_spectrum(src, M, Gt):
    """Route 2 with a spectrum from ``green_spectrum``; src is [Nz][Ny][Nx]."""
    s = _f64(src)
    N = _i64([s.shape[2], s.shape[1], s.shape[0]])
    MM = _i64(M)
    g = np.ascontiguousarray(Gt, dtype=np.complex128)
    phi = np.empty_like(s)
    rc = lib().oracle_solve_with_spectrum(_ptr(s), _ptr(N), _ptr(MM), _ptr(g), _ptr(phi))
    if rc:
        raise RuntimeError("oracle_solve_with_spectrum failed: %d" % rc)
    return phi


def solve(src, h, M=None):
    """Route 2 of the potential of ``src`` ([Nz][Ny][Nx], S = 4 pi rho) with
    cell widths h = (hx, hy, hz) on the doubled mesh M (default 2N)."""
    s = _f64(src)
    N = _i64([s.shape[2], s.shape[1], s.shape[0]])
    MM = _i64(doubled_mesh(N) if M is None else M)
    hh = _f64(h)
    phi = np.empty_like(s)
    rc = lib().oracle_solve(_ptr(s), _ptr(N), _ptr(MM), _ptr(hh), _ptr(phi))
    if rc:
        raise RuntimeError("oracle_solve failed: %d" % rc)
    return phi


def direct_sum(src, h):
    """Route 1: the discrete convolution with Eq. 6/9, summed cell by cell
    (O(N^6); meant for grids up to about 16^3-24^3)."""
    s = _f64(src)
    N = _i64([s.shape[2], s.shape[1], s.shape[0]])
    hh = _f64(h)
    phi = np.empty_like(s)
    lib().oracle_direct_sum(_ptr(s), _ptr(N), _ptr(hh), _ptr(phi))
    return phi


def direct_points(src, h, cells):
    """Route 1 at selected cells; ``cells`` are flat C-order indices into
    src.  O(N^3) per cell, so usable at full size for sampled checks."""
    s = _f64(src)
    N = _i64([s.shape[2], s.shape[1], s.shape[0]])
    hh = _f64(h)
    c = _i64(cells).ravel()
    out = np.empty(c.size, dtype=np.float64)
    lib().oracle_direct_points(_ptr(s), _ptr(N), _ptr(hh), _ptr(c), c.size, _ptr(out))
    return out


def max_rel_error(phi, ref):
    """Normwise max relative error, max|phi - ref| / max|ref|."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(phi - ref)) / np.max(np.abs(ref)))


def l1_error(phi, ref):
    """The L1 relative error norm of Sec. 4.1 (Eq. 11)."""
    phi = np.asarray(phi, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.sum(np.abs(phi - ref)) / np.sum(np.abs(ref)))
