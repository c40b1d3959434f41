"""GB300-native fast T-product of third-order quaternion tensors.

The compute path is the C-ABI library ``libqtp`` (hand-written CUDA for
sm_103a); ``paper_2212_14318_gb300.qtp`` is its thin ctypes binding.  Import
of this package loads nothing; the library is loaded on first use and a
missing or unbuilt library is an error (there is no CPU fallback).
"""
__all__ = ["qtp", "synth"]
