"""GB300-native five-equation RHS (WENO5-JS + HLLC + SSP-RK3) behind a C ABI.

The compute path is the CUDA library built from ``csrc/`` (``libmfc5.so``);
``mfc`` is its ctypes binding and ``inputs`` holds the seeded initial
conditions shared with the tests.
"""
