"""fgs4d: GB300-native 4D Gaussian Splatting rendering routine and its adjoint.

The compute path lives in ``csrc/`` (CUDA for sm_103a behind a C ABI); the
Python side only marshals arguments.  Submodules are imported lazily so that
``inputs`` can be used without loading the CUDA library.
"""
__all__ = ["inputs", "native", "render"]


def __getattr__(name):
    if name in __all__:
        import importlib
        return importlib.import_module(f"{__name__}.{name}")
    raise AttributeError(name)
