"""GB300-native loop-hafnian engine for Gaussian boson sampling (arXiv 2010.15595).

The compute path lives in CUDA kernels behind a C ABI (include/gbsh.h, libgbsh.so);
`paper_2010_15595_gb300.lib` is its Python binding.
"""
__all__ = ["lib", "workloads", "build"]
