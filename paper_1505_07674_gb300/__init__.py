"""GB300-native (sm_103a) ray-tracing likelihood for forward strong-lensing
reconstruction (Tessore, Bellagamba & Metcalf, "Lensed").

The compute path is the CUDA library built from ``csrc/`` (C ABI in
``include/lensed.h``); ``lensed.Model`` is its Python front end.
"""
__all__ = ["build", "lensed"]


def build(force=False):
    from ._build import build as _build

    return _build(force=force)
