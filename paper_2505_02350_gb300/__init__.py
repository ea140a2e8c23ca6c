"""SE-RBFNet optimisation hot path on GB300 (sm_103a).

The compute lives in libserbf.so (include/serbf.h); this package holds the
ctypes binding (``_native``), a device-resident problem wrapper (``field``),
the autograd wrapper (``autograd``) and the Algorithm 3 driver (``fitter``).
Importing a submodule that needs the library raises if it is not built.
"""
__all__ = ["_native", "field", "autograd", "fitter"]
