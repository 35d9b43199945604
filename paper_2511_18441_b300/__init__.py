"""B300-native region selection, recolouring and 3DGS rasterisation.

The compute path lives in the C-ABI library ``librecogs.so`` (hand-written
CUDA for sm_103a, declared in ``include/recogs.h``); ``binding`` marshals
torch tensors into its calls. ``scenegen`` draws seeded synthetic inputs.
Submodules are imported on first use so that input generation works
without a GPU.
"""
import importlib

__all__ = ["scenegen", "binding", "build"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
