"""GB300-native geometric adaptive smoothed aggregation (alpha-SA) multigrid
for DG discretisations: hand-written sm_103a CUDA kernels behind the C ABI
of include/gasa.h, and its Python binding (`gasa`)."""
from . import gasa  # noqa: F401
from .build import LIB, build  # noqa: F401
