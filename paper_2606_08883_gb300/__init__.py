"""libmrcm: GB300-native MRCM-OS-preconditioned flexible GMRES for Darcy pressure problems.

The compute path is the C-ABI shared library built from ``csrc/`` (hand-written CUDA for sm_103a);
``mrcm`` is the thin ctypes binding with the library's entry-point names.  ``workloads`` generates
seeded synthetic inputs.  Importing this package loads nothing; importing ``mrcm`` loads the
library and fails loudly if it has not been built.
"""
