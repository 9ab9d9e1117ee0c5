"""Torch-facing convenience over the C ABI: a ``Plan`` owns a library plan
and solves torch CUDA tensors on the caller's current stream.

PyTorch is used only for device memory and streams; every arithmetic step
of a solve runs in libisofft's kernels (through ``native``).
"""
import numpy as np
import torch

from . import native

# source / potential arrays: double for the FP64-class float-pair dtype too
_TORCH = {"f32": torch.float32, "f64": torch.float64, "df64": torch.float64}
_NUMPY = {"f32": np.float32, "f64": np.float64, "df64": np.float64}


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream


class Plan:
    """A solver for one mesh shape N = (Nx, Ny, Nz), widths h and dtype
    ('f32', 'f64', or 'df64' -- FP64-class float pairs on the FP32 units);
    sources and potentials are [Nz][Ny][Nx] arrays."""

    def __init__(self, n, h, dtype="f32", flags=0, verbosity=native.IPF_CONSOLE_ERROR, stream=None):
        if not torch.cuda.is_available():
            raise RuntimeError("isofft needs a CUDA device; there is no CPU path")
        self.n = tuple(int(v) for v in n)
        self.h = tuple(float(v) for v in h)
        self.dtype = dtype
        self.torch_dtype = _TORCH[dtype]
        self.handle = native.ipf_plan_create(self.n, self.h, dtype, flags, verbosity, _stream_handle(stream))

    @property
    def shape(self):
        return (self.n[2], self.n[1], self.n[0])

    @property
    def padded_shape(self):
        return native.ipf_plan_padded_shape(self.handle)

    @property
    def workspace_bytes(self):
        return native.ipf_plan_workspace_bytes(self.handle)

    @property
    def spectrum_bytes(self):
        return native.ipf_plan_spectrum_bytes(self.handle)

    def _check(self, t):
        if not (t.is_cuda and t.dtype == self.torch_dtype and t.is_contiguous() and tuple(t.shape) == self.shape):
            raise ValueError("expected a contiguous CUDA %s tensor of shape %s" % (self.torch_dtype, self.shape))

    def solve(self, src, out=None, stream=None):
        """Potential of `src` (S = 4 pi rho for gravity with G = 1).  `out`
        may be `src` itself.  Asynchronous on `stream` (default: current)."""
        self._check(src)
        if out is None:
            out = torch.empty_like(src)
        self._check(out)
        native.ipf_solve(self.handle, src.data_ptr(), out.data_ptr(), _stream_handle(stream))
        return out

    def solve_host(self, src, out=None, stream=None):
        """Solve from and to host numpy arrays (copies inside the call)."""
        src = np.ascontiguousarray(src, dtype=_NUMPY[self.dtype])
        if src.shape != self.shape:
            raise ValueError("source shape %s != %s" % (src.shape, self.shape))
        if out is None:
            out = np.empty_like(src)
        native.ipf_solve_host(self.handle, src.ctypes.data, out.ctypes.data, _stream_handle(stream))
        return out

    def solve_host_async(self, src, out, stream=None):
        """Enqueue a solve from host array `src` into host array `out`
        (numpy arrays or CPU torch tensors, pinned for asynchronous copies)
        and return at once; both must stay alive and untouched until
        host_wait()."""
        def ptr(a):
            return a.data_ptr() if hasattr(a, "data_ptr") else a.ctypes.data
        for a in (src, out):
            if tuple(a.shape) != self.shape:
                raise ValueError("array shape %s != %s" % (tuple(a.shape), self.shape))
        native.ipf_solve_host_async(self.handle, ptr(src), ptr(out), _stream_handle(stream))

    def host_wait(self):
        """Wait for every host solve enqueued on this plan."""
        native.ipf_plan_host_wait(self.handle)

    def pass_times(self):
        return native.ipf_plan_pass_times(self.handle)

    @property
    def variants(self):
        """(forward, inverse) y-pass forms: 0 tiles, 1 streamed."""
        return native.ipf_plan_variants(self.handle)

    def check(self, stream=None):
        """Synchronise the stream and raise if a bounded device wait of this
        plan's solves gave up since the previous check."""
        native.ipf_plan_check(self.handle, _stream_handle(stream))

    def close(self):
        if getattr(self, "handle", None):
            native.ipf_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def solve(src, h, out=None, stream=None):
    """One-off solve of a CUDA tensor; plans are not cached (use Plan)."""
    dtype = {torch.float32: "f32", torch.float64: "f64"}[src.dtype]
    nz, ny, nx = src.shape
    with Plan((nx, ny, nz), h, dtype, stream=stream) as p:
        return p.solve(src, out, stream)


def submit_batch(plans, srcs, outs, stream=None):
    """Enqueue independent solves of possibly different plans on one stream."""
    for p, s, o in zip(plans, srcs, outs):
        p._check(s)
        p._check(o)
    native.ipf_submit_batch([p.handle for p in plans], [s.data_ptr() for s in srcs],
                            [o.data_ptr() for o in outs], _stream_handle(stream))
    return outs


class BatchGraph:
    """A fixed batch of solves captured once into a CUDA graph.

    The batch's sources and outputs are the given tensors: refill the sources
    in place and ``replay()`` re-runs every solve (the library's internal
    streams appear in the graph as parallel branches).  The constructor runs
    the batch once outside capture so every one-off set-up (internal streams,
    kernel attributes) happens before the capture."""

    def __init__(self, plans, srcs, outs):
        self.plans, self.srcs, self.outs = list(plans), list(srcs), list(outs)
        submit_batch(self.plans, self.srcs, self.outs)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            submit_batch(self.plans, self.srcs, self.outs)
        torch.cuda.synchronize()

    def replay(self):
        self.graph.replay()
        return self.outs
