"""GB300-native NASGabor appearance evaluation (arXiv 2606.09794).

The compute path lives in the CUDA library ``libnasgabor.so`` (sources under
``csrc/``, C ABI in ``include/nasgabor.h``); ``binding`` is its thin Python
wrapper (ctypes marshalling of torch CUDA tensors) and ``inputs`` holds the
seeded synthetic workloads. Importing the package does not load the library;
``binding`` loads it on import and raises if it is missing.
"""
import importlib

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in __all__:
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
