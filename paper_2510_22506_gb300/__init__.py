"""GB300-native trace-regularized FCTN completion (PAM sweep) library.

The compute path is the C-ABI shared library ``libfctn.so`` built from
``csrc/``; ``fctn`` is its thin ctypes binding.  Importing the package does
not load the library; ``paper_2510_22506_gb300.fctn`` does, and fails loudly
if it has not been built.
"""
__all__ = ["fctn", "synth"]
