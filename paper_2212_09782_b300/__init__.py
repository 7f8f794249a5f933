"""QR-based TEBD bond update on B300 (sm_103a): Python binding of libqrtebd.

Importing the package loads nothing; ``paper_2212_09782_b300.lib`` loads the
CUDA library (and raises if it is missing: there is no CPU fallback).
"""
__all__ = ["lib", "workloads"]
