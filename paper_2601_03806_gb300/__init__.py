"""GB300 (sm_103a) ghost-mode filtered fluctuating lattice Boltzmann library.

The compute path is libflbm.so (CUDA kernels behind the C ABI of
include/flbm.h); ``flbm`` is its ctypes binding.  Accessing ``flbm``,
``Lattice`` or ``FlbmError`` fails loudly if the library has not been built
(``paper_2601_03806_gb300.build.build()`` builds it); there is no CPU path.
"""
import importlib

__all__ = ["flbm", "Lattice", "FlbmError", "build"]


def __getattr__(name):
    if name == "flbm":
        return importlib.import_module(".flbm", __name__)
    if name in ("Lattice", "FlbmError"):
        return getattr(importlib.import_module(".flbm", __name__), name)
    raise AttributeError(name)
