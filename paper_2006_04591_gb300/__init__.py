"""GB300-native digital shearlet transform (after tfShearlab, arXiv 2006.04591).

Submodules are imported lazily so that importing :mod:`synth` (the seeded
input generators) never loads the CUDA library.
"""

__all__ = ["synth", "shearlet", "autograd", "apps"]
