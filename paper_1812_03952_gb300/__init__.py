"""GB300-native CPR-FPF / FGMRES solver for thermal reservoir Jacobians.

The compute path is the CUDA library ``libtrs.so`` (C ABI declared in
``include/trs.h``); :mod:`.trs` is its thin ctypes binding and :mod:`.autograd`
the PyTorch autograd wrapper.  Importing this package loads nothing; the
library is loaded on first use and a missing library is an error.
"""
__all__ = ["synthetic", "trs", "autograd"]
