"""GB300 FED-FEM Pennes bio-heat library (Zhang & Chauhan, arXiv:1909.05098).

The compute path is the CUDA shared library built from csrc/ for sm_103a
(see :mod:`.build`); :mod:`.fedfem` is its ctypes binding.  Importing
:mod:`.fedfem` fails loudly if the library has not been built.
"""
__all__ = ["build", "fedfem"]
