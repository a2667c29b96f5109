"""Photon Field Networks (arXiv 2304.07338) hot path for B300 (sm_103a).

The compute path is libpf.so (CUDA kernels behind the C ABI of include/pf.h);
`api` is its thin torch binding.  Importing the package loads nothing: the
library is loaded on first use and a missing build raises.
"""
__all__ = ["api", "inputs", "build"]
