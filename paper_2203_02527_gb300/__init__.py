"""GB300-native 0th persistent homology barcodes (Rawson, arXiv 2203.02527).

The five steps of the paper's algorithm (Sec. 2; Sec. 4 steps 1-5) run as
hand-written CUDA kernels for sm_103a in libph0.so behind a C ABI
(include/ph0.h).  This package is the thin Python binding: `ph0` wraps the C
calls with torch tensors as device buffers, `inputs` generates the seeded
synthetic point clouds, `build` compiles the library.

Importing the package does not load the CUDA library; the first call does,
and fails loudly if it is missing.
"""

__all__ = ["ph0", "inputs", "build"]
