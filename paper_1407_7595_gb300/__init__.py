"""GB300-native matrix-element-method integrator (arXiv:1407.7595 hot path).

The compute path is the C-ABI CUDA library ``libmem.so`` (sources in ``csrc/``,
declarations in ``include/mem.h``); ``abi`` is its thin ctypes binding and
``synth`` the seeded synthetic-input generators. Importing this package does
not load the CUDA library; ``abi.lib()`` does, and fails loudly if it is missing.
"""
__all__ = ["abi", "synth"]
