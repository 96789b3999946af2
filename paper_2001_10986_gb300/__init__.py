"""GB300 implementation of entropic domain decomposition for optimal transport.

The compute path is the CUDA library built from csrc/ (C ABI in include/dd.h);
`paper_2001_10986_gb300.dd` is its Python binding. `synthetic` provides
seeded problem data.
"""
__all__ = ["dd", "synthetic", "build"]
