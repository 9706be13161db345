"""GB300-native closed-shell CCSD(T) triples-correction energy.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``, declared in ``include/tcorr.h``); ``tcorr`` is its thin
ctypes binding.  ``synth`` generates seeded synthetic inputs.
"""
__all__ = ["synth", "tcorr"]


def __getattr__(name):
    if name == "tcorr":
        from . import tcorr as mod
        return mod
    if name == "synth":
        from . import synth as mod
        return mod
    raise AttributeError(name)
