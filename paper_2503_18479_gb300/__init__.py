"""GB300-native (sm_103a) differentiable forward map C -> Bz of capacitively tuned loop
arrays, with adjoint gradients.

Layout:
  include/mts.h (repo root)  C ABI
  csrc/                      CUDA kernels and the C ABI implementation (libmts.so)
  native.py                  ctypes binding, one function per ABI entry point
  simulator.py               Simulator + torch.autograd.Function
  workloads.py               seeded synthetic inputs (no method arithmetic)
  build_lib.py               nvcc build of lib/libmts.so

Importing the package does not load the CUDA library; the first call does, and fails
loudly if the library was not built.
"""
__all__ = ["Simulator", "MtsFunction", "native", "workloads"]


def __getattr__(name):
    if name in ("Simulator", "MtsFunction"):
        from . import simulator
        return getattr(simulator, name)
    raise AttributeError(name)
