"""B300-native region selection, recolouring and 3DGS rasterisation.

The compute path lives in the C-ABI library ``librecogs.so`` (hand-written
CUDA for sm_103a, declared in ``include/recogs.h``); ``binding`` marshals
torch tensors into its calls. ``scenegen`` draws seeded synthetic inputs.
The binding is imported lazily so that input generation works without a GPU.
"""

__all__ = ["scenegen", "binding"]


def __getattr__(name):
    if name == "binding":
        from . import binding
        return binding
    raise AttributeError(name)
