"""GB300-native batched enhanced normalized min-sum decoding of short BCH codes.

Implements the decoder of arXiv 2412.20828 (Li & Yu, "Effective Application of
Normalized Min-Sum Decoding for Short BCH Codes") as a C-ABI library over
hand-written sm_103a CUDA kernels; ``bchdec`` is the thin ctypes binding.
Importing the package does not load the library; ``bchdec`` does, and fails loudly
when it has not been built.
"""
__all__ = ["bchdec", "synth"]
