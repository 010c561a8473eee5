"""GB300-native periodic 1D heat stencil (arXiv 2307.01117, Section 2, Eq. 2).

The compute path is hand-written CUDA for sm_103a behind the C ABI declared in
``include/heat.h`` (``libheat.so``); ``heat`` is the ctypes binding.
"""
