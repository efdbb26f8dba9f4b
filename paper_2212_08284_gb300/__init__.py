"""GB300-native ANKH: interpolated-Ewald energy and forces of periodic point
multipoles (charges, dipoles, quadrupoles) behind a small C ABI.

The compute path lives in ``csrc/`` (CUDA for sm_103a, built into
``libankh.so``); ``api`` is a thin ctypes binding plus a
``torch.autograd.Function``.  ``synth`` draws the seeded synthetic workloads.
"""
__all__ = ["api", "synth"]
