"""GB300-native quantum quasi-Monte Carlo (QQMC) for the Anderson dot.

The computation lives in the CUDA library built from ``csrc/`` (C ABI in
``include/qqmc.h``); ``qqmc`` is its ctypes binding, ``workloads`` draws the
seeded synthetic inputs and ``build`` compiles the library for sm_103a.
Nothing here falls back to the CPU.
"""
__all__ = ["qqmc", "workloads", "build"]
