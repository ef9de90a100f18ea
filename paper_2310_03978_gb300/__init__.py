"""GB300-native sliced tensor-network contraction for random-circuit amplitudes.

Submodules are imported on demand: ``workload`` (seeded inputs, no device code) and
``tn`` (the binding to the C-ABI library ``libtn.so``).
"""
__all__ = ["workload", "tn"]
