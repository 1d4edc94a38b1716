"""GB300-native TNMCMC-1 slice update (arXiv 2509.23945).

``inputs``  seeded synthetic lattices and chain layouts (no method arithmetic)
``tnmc``    ctypes binding of the CUDA library (C ABI in include/tnmc.h)
``build_lib`` builds the library for sm_103a
"""

__all__ = ["inputs", "tnmc", "build_lib"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
