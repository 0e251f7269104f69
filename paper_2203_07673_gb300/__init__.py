"""GB300-native FusedMM: an SDDMM feeding an SpMM in one CUDA kernel.

``fmm``       the binding of the C ABI (include/fmm.h) in libfmm.so
``autograd``  FusedMM as a differentiable op with a hand-written adjoint
``workloads`` seeded synthetic inputs shaped like the paper's workloads
``build``     compiles libfmm.so in-tree with nvcc (sm_103a)

Submodules are imported on use, so ``workloads`` needs neither a GPU nor the
built library.
"""
import importlib

__all__ = ["fmm", "autograd", "workloads", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
