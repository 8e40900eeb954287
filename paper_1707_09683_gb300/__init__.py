"""GB300-native MSV/SSV protein-profile scan library.

The compute path is a C-ABI shared library (``csrc/``, declared in
``include/mpf.h``) of hand-written sm_103a CUDA kernels; ``mpf`` is its thin
ctypes binding, ``synth`` the seeded input generator.  Importing the package
loads nothing; ``paper_1707_09683_gb300.mpf`` loads the library on first use
and raises if it is missing.
"""
__all__ = ["mpf", "synth"]
