"""GB300-native multinomial-logit Newton-Raphson (Hasan, Wang & Mahani, arXiv:1404.3177).

The compute path is the CUDA library ``_lib/libmnl.so`` (C ABI in
``include/mnl.h``); this package marshals torch tensors into it.  PyTorch only
provides device memory and the current CUDA stream.

    import torch
    from paper_1404_3177_gb300 import MNL
    m = MNL(X, Y, Z, choice, precision="bf16")      # cuda tensors
    theta, info = m.fit()                            # float64 cuda tensor

``datagen`` (seeded synthetic problems) needs neither torch nor the library.
"""
from __future__ import annotations

__all__ = ["MNL", "build", "native"]


def build(force: bool = False) -> str:
    from . import _build
    return _build.build(force=force)


def __getattr__(name):
    if name == "MNL":
        from .api import MNL
        return MNL
    if name == "native":
        from . import _native
        return _native
    raise AttributeError(name)
