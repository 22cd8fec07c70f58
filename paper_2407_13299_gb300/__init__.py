"""Density-matrix purification with Ozaki-scheme products on GB300 (sm_103a).

The computation lives in libdmp.so (CUDA kernels behind the C ABI of
include/dmp.h); `paper_2407_13299_gb300.dmp` is its thin Python binding and
`paper_2407_13299_gb300.build` compiles it. Importing this package loads
nothing; the library is loaded on the first call into `dmp`.
"""

__all__ = ["build", "dmp"]
