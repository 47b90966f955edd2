"""GB300-native construction of spiking-network connectivity in GPU memory.

The compute path is the CUDA library libsnc.so (hand-written sm_103a kernels
behind the C ABI declared in include/snc.h); `paper_2306_09855_gb300.snc` is
its thin ctypes binding.  Importing the package itself loads nothing, so that
the seeded workload definitions in `workloads` stay usable without a GPU.
"""
__all__ = ["snc", "workloads"]
