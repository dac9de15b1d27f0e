"""hx27: wavelength-adaptive 27-point Helmholtz operator and solver for GB300.

The compute path lives in the C-ABI shared library built from ``csrc/``
(declared in ``include/hx27.h``); ``binding`` marshals arguments to it with
ctypes.  ``synth`` draws seeded synthetic inputs.  Importing this package does
not load the library; ``binding.lib()`` does, and raises if it is missing.
"""
__all__ = ["binding", "synth"]
