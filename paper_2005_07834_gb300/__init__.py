"""Local real-space RPA screening (chi0 and W on site grids) for GB300.

The compute path lives in the CUDA library ``liblrs.so`` (C-ABI, declared in
``include/lrs.h``); ``lrs`` is its ctypes binding and ``autograd`` wraps the
forward build and the adjoint kernel as a torch.autograd.Function.  Importing
this package loads nothing; the library is opened on first use and its absence
is an error, never a fallback.
"""
__all__ = ["synth", "lrs", "autograd"]
