"""GB300-native (sm_103a) QV-Tree Search: the data-parallel hot path of
"Stochastic 2-D Motion Planning with a POMDP Framework" (Sun and Kumar).

The computation lives in libqvts.so (C ABI: include/qvts.h); this package is
its thin Python binding plus the seeded workload generators.
"""
from . import workloads  # noqa: F401

__version__ = "0.1.0"


def __getattr__(name):
    # the binding imports torch and loads libqvts.so on first use
    if name in ("api", "_native", "autograd"):
        import importlib
        return importlib.import_module(f".{name}", __name__)
    raise AttributeError(name)
