"""B300-native (sm_103a) Tamm-Dancoff BSE hot path: W(q) interpolation, LRI pair
projection, H assembly and Haydock spectrum behind the C ABI of include/bse.h.

The compute path is the CUDA library libbse.so in this directory; this package only
binds it.  Importing :mod:`paper_2607_05853_b300.api` fails loudly when the library
has not been built.
"""
__all__ = ["api", "build"]
