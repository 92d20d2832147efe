"""GB300-native 2D Gaussian (surfel) splatting rasterizer hot path of
CityGaussianV2 (arXiv 2411.00771): CUDA kernels for sm_103a behind a C ABI
(``libgs2d.so``), with a thin ctypes binding in :mod:`.binding`.

Importing the package loads nothing; :mod:`.binding` loads the compiled
library and fails loudly when it is missing.
"""
__all__ = ["binding", "synthetic"]
