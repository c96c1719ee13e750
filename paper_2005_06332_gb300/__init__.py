"""GB300-native multi-morphology neuron stepper (HH + Hines tree solve).

The compute path lives in the CUDA library built from ``csrc/`` and is
reached through ``mm`` (a ctypes binding of the C-ABI in ``include/mm.h``).
Importing this package loads nothing native; ``mm`` loads the library on
first use and raises if it is missing.
"""
__all__ = ["netgen", "mm"]
