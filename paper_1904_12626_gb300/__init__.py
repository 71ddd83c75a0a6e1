"""GB300-native matrix profile (all-pairs z-normalised similarity join).

The compute path is the CUDA library ``libmpgb.so`` built from ``csrc/``;
this package only marshals arguments to its C entry points.  The library is
loaded on first use, and every call fails loudly if it is missing.
"""
