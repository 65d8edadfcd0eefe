"""B300-native hot path of the explicit electromagnetic PIC timestep (lambdaPIC).

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI, header
``include/lpic.h``); ``lpic`` is its thin ctypes binding.
"""
