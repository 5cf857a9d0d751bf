"""GB300-native fictitious-wave CSEM gradient engine (Yang, arXiv 2211.16665).

The hot path -- leap-frog Yee stepping with CPML fused with the damped
on-the-fly transform, adjoint runs driven by basis-function adjoint sources,
and the resistivity gradient -- runs in the CUDA library `libcsemfw.so`
behind the C ABI of `include/csem.h`.  This package holds the ctypes binding
(`_capi`), a torch-facing wrapper (`engine`), the autograd Function
(`autograd`), the native build (`_build`) and the seeded synthetic inputs
(`workloads`).
"""
__all__ = ["workloads"]
