"""GB300-native NASGabor appearance evaluation (arXiv 2606.09794).

The compute path lives in the CUDA library ``libnasgabor.so`` (sources under
``csrc/``, C ABI in ``include/nasgabor.h``); ``binding`` is its thin Python
wrapper (ctypes marshalling of torch CUDA tensors) and ``inputs`` holds the
seeded synthetic workloads. Importing the package does not load the library;
``binding`` loads it on import and raises if it is missing.
"""

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name == "binding":
        from . import binding
        return binding
    if name == "inputs":
        from . import inputs
        return inputs
    raise AttributeError(name)
