"""GB300-native optimiser of the Gaussian-LIC photo-realistic map (arXiv 2404.06926).

The compute path is a CUDA library (``csrc/``, sm_103a) behind a C ABI declared
in ``include/gl_map.h``; ``binding`` marshals arguments to it with ctypes.
Importing this package loads nothing; ``binding.lib()`` loads the library and
raises if it has not been built.
"""
__all__ = ["scenes"]
