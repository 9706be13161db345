"""GB300-native closed-shell CCSD(T) triples-correction energy.

The compute path is a C-ABI shared library of hand-written sm_103a CUDA
kernels (``csrc/``, declared in ``include/tcorr.h``); ``tcorr`` is its thin
ctypes binding (``from paper_1609_08094_gb300 import tcorr``).  ``synth``
generates seeded synthetic inputs.
"""
__all__ = ["synth", "tcorr"]
