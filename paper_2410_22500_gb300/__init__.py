"""GB300-native fast hyperspectral reconstruction (arXiv 2410.22500).

The compute path lives in the C-ABI library libfhr.so (hand-written CUDA for
sm_103a, declared in include/fhr.h); `paper_2410_22500_gb300.fhr` is its thin
ctypes binding and `paper_2410_22500_gb300.synth` draws seeded inputs.
Importing the package loads nothing; the library is loaded on first use and
a missing library is an error (there is no CPU fallback).
"""
__all__ = ["fhr", "synth"]
