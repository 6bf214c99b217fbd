"""IBIP on one GB300 GPU: image-based invasion percolation (Gostick, Yang &
Boek, arXiv 2101.03240) as hand-written CUDA kernels behind a C ABI
(include/ibip.h), with a thin PyTorch/ctypes binding (``ibip``) and seeded
synthetic inputs (``synth``)."""

__all__ = ["ibip", "synth", "build_lib"]
