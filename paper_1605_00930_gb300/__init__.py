"""GB300-native IWPP morphological reconstruction (reconstruction by dilation and
fill-holes / reconstruction by erosion) behind a small C ABI.

The binding (``paper_1605_00930_gb300.iwpp``) is imported lazily so that the
input generators in ``synth`` can be used without loading the CUDA library.
"""
import importlib

__all__ = ["iwpp", "synth"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
