"""GB300-native isolated-system Poisson solver (Hockney's mesh doubling in
3-D as in Budiardja & Cardall's PSPFFT).

* ``native``  -- ctypes binding of the C ABI (include/isofft.h), same names.
* ``solver``  -- ``Plan`` / ``solve`` / ``submit_batch`` on torch CUDA tensors.
* ``sources`` -- seeded synthetic source distributions (shared with tests).
* ``build``   -- compiles libisofft.so for sm_103a.

Importing the package loads nothing; the CUDA library is built/loaded at the
first call and every entry point raises if it is unavailable.
"""

__all__ = ["native", "solver", "sources", "build", "Plan", "solve", "submit_batch", "BatchGraph"]


def __getattr__(name):
    if name in ("Plan", "solve", "submit_batch", "BatchGraph"):
        from . import solver
        return getattr(solver, name)
    if name in ("native", "solver", "sources", "build"):
        import importlib
        return importlib.import_module("." + name, __name__)
    raise AttributeError(name)
