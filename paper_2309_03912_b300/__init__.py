"""B300-native transform-reduce-scan over "hdc" maps (libtr).

The compute lives in ``libtr.so`` (hand-written CUDA for sm_103a, C ABI in
``include/tr.h``); ``binding`` marshals torch tensors into those calls and
``inputs`` draws the seeded synthetic workloads.  Importing this package does
not load the library; the first call through ``binding`` does, and raises if
it has not been built (``python -m paper_2309_03912_b300.build``).
"""
__all__ = ["binding", "inputs", "build"]
