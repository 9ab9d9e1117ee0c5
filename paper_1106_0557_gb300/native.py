"""ctypes binding of the C ABI in include/isofft.h.

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  The functions carry the C names; a non-zero status raises
``IsofftError``.  Pointers are plain integers (``tensor.data_ptr()``,
``numpy.ndarray.ctypes.data``), streams are ``cudaStream_t`` values as
integers (``torch.cuda.current_stream().cuda_stream``), 0 for the default
stream.

There is no CPU fallback: if ``libisofft.so`` cannot be built or loaded,
every entry point raises.
"""
import ctypes
import os

from . import build as _build

IPF_F32 = 0
IPF_F64 = 1
IPF_DF64 = 2
IPF_OK = 0
IPF_INVALID_ARG = 1
IPF_UNSUPPORTED_SIZE = 2
IPF_OUT_OF_MEMORY = 3
IPF_CUDA_ERROR = 4
IPF_TIMEOUT = 5
IPF_BUDGET_EXCEEDED = 6
IPF_NOT_READY = 7
IPF_CONSOLE_ERROR = 0
IPF_CONSOLE_WARNING = 1
IPF_CONSOLE_INFO_1 = 2
IPF_CONSOLE_INFO_2 = 3
IPF_FLAG_PASS_EVENTS = 1
IPF_FLAG_Y_TILES = 2
IPF_FLAG_Y_STREAM = 4
IPF_FLAG_TEST_WAIT_RUNOUT = 8
IPF_FLAG_TEST_CANARY = 16
IPF_FLAG_Y_TILES_NARROW = 32

DTYPES = {"f32": IPF_F32, "f64": IPF_F64, "df64": IPF_DF64, IPF_F32: IPF_F32, IPF_F64: IPF_F64,
          IPF_DF64: IPF_DF64}

_lib = None


class IsofftError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        super().__init__("%s: %s (status %d)" % (where, status_string(status), status))


def _declare(L):
    vp, i64p = ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64)
    dp = ctypes.POINTER(ctypes.c_double)
    sig = {
        "ipf_plan_create": [ctypes.POINTER(vp), i64p, dp, ctypes.c_int, ctypes.c_uint32, ctypes.c_int, vp],
        "ipf_plan_destroy": [vp],
        "ipf_plan_padded_shape": [vp, i64p],
        "ipf_plan_workspace_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
        "ipf_plan_spectrum_bytes": [vp, ctypes.POINTER(ctypes.c_size_t)],
        "ipf_estimate_bytes": [i64p, dp, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)],
        "ipf_solve": [vp, vp, vp, vp],
        "ipf_solve_host": [vp, vp, vp, vp],
        "ipf_solve_host_async": [vp, vp, vp, vp],
        "ipf_plan_host_wait": [vp],
        "ipf_solve_noalloc": [i64p, dp, ctypes.c_int, vp, vp, vp],
        "ipf_plan_check": [vp, vp],
        "ipf_plan_variants": [vp, ctypes.POINTER(ctypes.c_int)],
        "ipf_noalloc_check": [vp],
        "ipf_submit_batch": [ctypes.POINTER(vp), ctypes.c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), vp],
        "ipf_plan_pass_times": [vp, ctypes.POINTER(ctypes.c_float)],
        "ipf_greens_cache_bytes": [ctypes.POINTER(ctypes.c_size_t)],
        "ipf_greens_cache_trim": [ctypes.c_size_t],
        "ipf_launch_count": [ctypes.POINTER(ctypes.c_uint64)],
        "ipf_last_cuda_error": [],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    L.ipf_status_string.argtypes = [ctypes.c_int]
    L.ipf_status_string.restype = ctypes.c_char_p
    return L


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libisofft.so, building it first if it is missing or stale."""
    global _lib
    if _lib is None:
        path = _build.build()
        if not os.path.exists(path):
            raise RuntimeError("libisofft.so is missing and could not be built")
        _lib = _declare(ctypes.CDLL(path))
    return _lib


def status_string(status: int) -> str:
    return ipf_status_string(status)


def ipf_status_string(status: int) -> str:
    return lib().ipf_status_string(int(status)).decode()


def _check(rc, where):
    if rc != IPF_OK:
        raise IsofftError(rc, where)


def _i64x3(v):
    return (ctypes.c_int64 * 3)(*[int(x) for x in v])


def _f64x3(v):
    return (ctypes.c_double * 3)(*[float(x) for x in v])


def ipf_plan_create(n, h, dtype="f32", flags=0, verbosity=IPF_CONSOLE_ERROR, stream=0):
    out = ctypes.c_void_p()
    rc = lib().ipf_plan_create(ctypes.byref(out), _i64x3(n), _f64x3(h), DTYPES[dtype], int(flags),
                               int(verbosity), ctypes.c_void_p(int(stream)))
    _check(rc, "ipf_plan_create")
    return out.value


def ipf_plan_destroy(plan):
    _check(lib().ipf_plan_destroy(ctypes.c_void_p(plan)), "ipf_plan_destroy")


def ipf_plan_padded_shape(plan):
    m = (ctypes.c_int64 * 3)()
    _check(lib().ipf_plan_padded_shape(ctypes.c_void_p(plan), m), "ipf_plan_padded_shape")
    return tuple(int(x) for x in m)


def ipf_plan_workspace_bytes(plan):
    b = ctypes.c_size_t()
    _check(lib().ipf_plan_workspace_bytes(ctypes.c_void_p(plan), ctypes.byref(b)), "ipf_plan_workspace_bytes")
    return int(b.value)


def ipf_plan_spectrum_bytes(plan):
    b = ctypes.c_size_t()
    _check(lib().ipf_plan_spectrum_bytes(ctypes.c_void_p(plan), ctypes.byref(b)), "ipf_plan_spectrum_bytes")
    return int(b.value)


def ipf_estimate_bytes(n, h, dtype="f32"):
    b = ctypes.c_size_t()
    _check(lib().ipf_estimate_bytes(_i64x3(n), _f64x3(h), DTYPES[dtype], ctypes.byref(b)), "ipf_estimate_bytes")
    return int(b.value)


def ipf_solve(plan, d_src, d_phi, stream=0):
    _check(lib().ipf_solve(ctypes.c_void_p(plan), ctypes.c_void_p(int(d_src)), ctypes.c_void_p(int(d_phi)),
                           ctypes.c_void_p(int(stream))), "ipf_solve")


def ipf_solve_host(plan, h_src, h_phi, stream=0):
    _check(lib().ipf_solve_host(ctypes.c_void_p(plan), ctypes.c_void_p(int(h_src)), ctypes.c_void_p(int(h_phi)),
                                ctypes.c_void_p(int(stream))), "ipf_solve_host")


def ipf_plan_check(plan, stream=0):
    """Synchronise `stream`; raise IsofftError if a bounded device wait of
    the plan's solves gave up since the previous check."""
    _check(lib().ipf_plan_check(ctypes.c_void_p(plan), ctypes.c_void_p(int(stream))), "ipf_plan_check")


def ipf_plan_variants(plan):
    """(forward, inverse) y-pass forms of a plan: 0 tiles, 1 streamed."""
    v = (ctypes.c_int * 2)()
    _check(lib().ipf_plan_variants(ctypes.c_void_p(plan), v), "ipf_plan_variants")
    return int(v[0]), int(v[1])


def ipf_noalloc_check(stream=0):
    _check(lib().ipf_noalloc_check(ctypes.c_void_p(int(stream))), "ipf_noalloc_check")


def ipf_solve_host_async(plan, h_src, h_phi, stream=0):
    _check(lib().ipf_solve_host_async(ctypes.c_void_p(plan), ctypes.c_void_p(int(h_src)),
                                      ctypes.c_void_p(int(h_phi)), ctypes.c_void_p(int(stream))),
           "ipf_solve_host_async")


def ipf_plan_host_wait(plan):
    _check(lib().ipf_plan_host_wait(ctypes.c_void_p(plan)), "ipf_plan_host_wait")


def ipf_solve_noalloc(n, h, dtype, d_src, d_phi, stream=0):
    """Plan-free solve whose scratch is the library's static device array
    (no allocation); see include/isofft.h for its limits."""
    _check(lib().ipf_solve_noalloc(_i64x3(n), _f64x3(h), DTYPES[dtype], ctypes.c_void_p(int(d_src)),
                                   ctypes.c_void_p(int(d_phi)), ctypes.c_void_p(int(stream))), "ipf_solve_noalloc")


def ipf_submit_batch(plans, d_srcs, d_phis, stream=0):
    n = len(plans)
    if len(d_srcs) != n or len(d_phis) != n:
        raise ValueError("plans, sources and outputs differ in length")
    P = (ctypes.c_void_p * n)(*plans)
    S = (ctypes.c_void_p * n)(*[int(p) for p in d_srcs])
    O = (ctypes.c_void_p * n)(*[int(p) for p in d_phis])
    _check(lib().ipf_submit_batch(P, n, S, O, ctypes.c_void_p(int(stream))), "ipf_submit_batch")


def ipf_plan_pass_times(plan):
    ms = (ctypes.c_float * 5)()
    _check(lib().ipf_plan_pass_times(ctypes.c_void_p(plan), ms), "ipf_plan_pass_times")
    return [float(x) for x in ms]


def ipf_greens_cache_bytes():
    b = ctypes.c_size_t()
    _check(lib().ipf_greens_cache_bytes(ctypes.byref(b)), "ipf_greens_cache_bytes")
    return int(b.value)


def ipf_greens_cache_trim(budget):
    _check(lib().ipf_greens_cache_trim(int(budget)), "ipf_greens_cache_trim")


def ipf_launch_count():
    c = ctypes.c_uint64()
    _check(lib().ipf_launch_count(ctypes.byref(c)), "ipf_launch_count")
    return int(c.value)


def ipf_last_cuda_error():
    return int(lib().ipf_last_cuda_error())
