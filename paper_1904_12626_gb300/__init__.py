"""GB300-native matrix profile (all-pairs z-normalised similarity join).

The compute path is the CUDA library ``libmpgb.so`` built from ``csrc/``
(``build.build()``); ``api`` only marshals PyTorch tensors to its C entry
points (declared in ``include/mp.h``).  The library is loaded on first use
and every call fails loudly if it is missing.

    from paper_1904_12626_gb300 import selfjoin, abjoin, batched, pan, matrix_profile

``tune.Tuner`` chooses each call's tile configuration by measurement.
"""
_API = ("selfjoin", "selfjoin_lr", "abjoin", "batched", "pan", "stats", "backward",
        "matrix_profile", "MatrixProfileFn", "Anytime", "fluss", "device_status", "init",
        "profile_length", "exclusion_zone", "workspace")


def __getattr__(name):
    if name in _API:
        from . import api
        return getattr(api, name)
    if name == "Tuner":
        from .tune import Tuner
        return Tuner
    raise AttributeError(name)
