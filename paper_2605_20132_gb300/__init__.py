"""GB300-native chunked DAS filter chain (FiLark's streaming operator chain).

The product is libfilark (CUDA for sm_103a behind the C-ABI in
include/filark.h).  ``abi`` is the ctypes binding with the C names, ``chain``
a PyTorch-friendly wrapper, ``synth`` the seeded synthetic input streams.
"""
