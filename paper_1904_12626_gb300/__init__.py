"""GB300-native matrix profile (all-pairs z-normalised similarity join).

The compute path is the CUDA library ``libmpgb.so`` built from ``csrc/``
(``build.build()``); ``api`` only marshals PyTorch tensors to its C entry
points (declared in ``include/mp.h``).  The library is loaded on first use
and every call fails loudly if it is missing.

    from paper_1904_12626_gb300 import selfjoin, abjoin, batched, pan, matrix_profile
"""
_API = ("selfjoin", "abjoin", "batched", "pan", "stats", "backward", "matrix_profile",
        "MatrixProfileFn", "device_status", "init", "profile_length", "exclusion_zone",
        "workspace")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    raise AttributeError(name)
