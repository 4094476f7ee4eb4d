"""GB300-native FFT Lindhard susceptibility (Wang et al., Sec. 2 Eq. 9, Sec. 3).

The compute path is the CUDA library built from ``csrc/`` (``liblindhard.so``)
and reached through the C ABI declared in ``include/lindhard.h``; the Python
module ``lindhard`` only marshals arguments to it.
"""
