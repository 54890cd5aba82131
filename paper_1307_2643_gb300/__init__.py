"""GB300-native propagation of cosmic-ray candidates through gridded magnetic
fields (the module / candidate / IsActive method of CRPropa 3.0,
arXiv:1307.2643).

The compute path is the CUDA library ``_build/libcrp.so`` (sources in
``csrc/``, C ABI in ``include/crp.h``, built by ``build.build()``); ``crp``
is its ctypes binding.
"""
from . import crp  # noqa: F401

__all__ = ["crp"]
