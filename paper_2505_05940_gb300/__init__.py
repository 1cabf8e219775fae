"""GB300-native differentiable modal synthesis of nonlinear strings, membranes
and plates (Diaz & Sandler, DAFx25): C-ABI CUDA library + thin Python binding.

    physics    modes, projections and excitation of the library's plan step
    coupling   von Karman coupling tensors of simply supported rectangles
    _native    ctypes binding of libmdx.so (include/mdx.h)
    modal      high-level API: build instances, simulate, gradients (autograd)
    workloads  seeded synthetic physical parameters (shared with the tests)
"""
__all__ = ["physics", "coupling", "modal", "workloads"]
