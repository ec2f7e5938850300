"""GB300-native stellar-disk integration (SOAP-GPU hot path, arXiv 2301.04259).

The compute path lives in the CUDA shared library built from ``csrc/`` and is
reached through ``paper_2301_04259_gb300.soap`` (a ctypes binding with the
same names as the C-ABI in ``include/soap.h``).  ``synth`` holds the seeded
synthetic-input generators; it carries none of the method's arithmetic.

Importing this package does not load the CUDA library; ``soap`` does, and it
raises if the library has not been built.
"""

__all__ = ["soap", "synth"]
