"""GB300-native Elfpie gradient step (arXiv 2209.14671).

The compute path is the C-ABI library ``libelfpie.so`` built from ``csrc/``
(hand-written sm_103a CUDA); ``elfpie`` is its thin ctypes binding.  Importing
this package does not load the library; ``elfpie.load()`` does, and fails loudly
when it is missing.
"""
__all__ = ["inputs", "elfpie"]
