"""GB300-native butterfly sparse Fourier transform (Ying, "Sparse Fourier Transform via
Butterfly Algorithm").  The compute path is libbfly.so (csrc/, C ABI in include/bfly.h);
this package only marshals arguments.  Importing it does not load the library; the first
Plan does, and raises if the library is missing or unusable."""
import importlib

__all__ = ["Plan", "Batch", "butterfly", "butterfly_fn", "measure_peak", "ShardLayout", "ShardedTransform",
           "FarField"]
_WHERE = {"ShardLayout": ".sharded", "ShardedTransform": ".sharded", "FarField": ".farfield"}


def __getattr__(name):
    if name in __all__:
        return getattr(importlib.import_module(_WHERE.get(name, ".plan"), __name__), name)
    raise AttributeError(name)
