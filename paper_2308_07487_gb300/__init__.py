"""GB300-native spin pair correlation (arXiv 2308.07487): C-ABI library + thin binding.

The compute path lives in ``csrc/`` (CUDA for sm_103a) behind the C-ABI declared in
``include/asd.h``; ``asd`` (the ctypes binding) only marshals arguments.  Importing
this package does not load the library: ``from paper_2308_07487_gb300 import asd``
does, and fails loudly if it has not been built.
"""
__all__ = ["asd", "synth"]
