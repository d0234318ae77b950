"""GB300-native differentiable Gaussian-splatting rasteriser (S3PO-GS hot path).

The compute path is the CUDA library ``libs3gs.so`` built from ``csrc/`` for
sm_103a; ``binding`` wraps its C ABI (declared in ``include/s3gs.h``) and
``autograd`` exposes it to PyTorch. Submodules are imported lazily so that the
seeded scene generators can be used without loading the CUDA library.
"""
import importlib

__all__ = ["scenes", "binding", "autograd", "autotune", "build", "slam"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
