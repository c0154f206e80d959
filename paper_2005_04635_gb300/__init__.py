"""GB300-native Grover state-vector simulator (arXiv 2005.04635, equivalent
operator method).

The compute path is ``libgrover.so`` (hand-written CUDA for sm_103a behind a C
ABI, declared in ``include/grover.h``); ``binding`` marshals arguments to it
from torch tensors and streams.  Importing this package does not load the
library; the first call into ``binding`` does, and raises if it is missing.
"""

__all__ = ["binding", "inputs"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
