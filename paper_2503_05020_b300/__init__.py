"""B300-native multi-environment IPC stepper (GRIP, arXiv 2503.05020): C ABI + Python binding.

`ipc.Scene` drives the sm_103a kernels of libipc_b300.so; `scenes` builds seeded synthetic
grasp environments. Nothing here computes the method on the CPU.
"""
from . import scenes  # noqa: F401

__all__ = ["scenes", "ipc", "build"]
